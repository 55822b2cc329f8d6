"""GPU exact step (App. C: convection of the composition fields and the
Fletcher-Reeves inversion omega~ = Phi^{-1}(Phi~)) against the FP64 oracle:
fixed iteration counts (PLAIN_FP64, element by element), convergence to the
tolerance (iteration counts and states), the MIXED_FP32 differential paths, the
reduction to the truncated step, batches and error handling."""
import numpy as np
import pytest

import oracle as O
import paper_1804_02883_gb300 as P
from paper_1804_02883_gb300 import workloads as W
from helpers import fluct_err, oracle_params, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build(oracle_lib):
    P.lib()


def _random_state(ny, nx, seed, vamp):
    return (W.random_omega(ny, nx, seed=seed, amp=0.05), W.random_populations(ny, nx, seed=seed + 1),
            W.random_velocity(ny, nx, seed=seed + 2, amp=vamp))


def _oracle_exact(r, omega, pop, vel, max_iter, tol, nsteps=1):
    p = oracle_params(r)
    phi, q = O.solve(p, omega)
    st = O.State(omega.copy(), pop.copy(), vel.copy(), phi, q, np.zeros((2, r.ny, r.nx)))
    stats = O.step_exact(p, st, nsteps, max_iter=max_iter, tol=tol)
    return st, stats


@pytest.mark.parametrize("ny,nx,ns,iters", [(32, 32, 8, 4), (16, 64, 8, 2), (64, 32, 12, 6)])
def test_exact_step_fp64_fixed_iterations(ny, nx, ns, iters):
    r = P.RunParams(nx=nx, ny=ny, ns=ns, precision=P.PLAIN_FP64, f_a=0.5, phi_p=0.2, f0=10.0)
    omega, pop, vel = _random_state(ny, nx, 31, 0.02)
    h = P.EpdLb([r])
    h.set_state(0, omega, pop, vel)
    h.set_inversion(iters, 0.0)
    h.step(1)
    h.sync()
    st, stats = _oracle_exact(r, omega, pop, vel, iters, 0.0)
    s = h.inversion_stats(0)
    assert s["iterations"] == iters == int(stats[0, 0])
    assert abs(s["residual0"] - stats[0, 1]) <= 1e-12 * stats[0, 1]
    assert abs(s["residual"] - stats[0, 2]) <= 1e-8 * stats[0, 2]
    gom, gpop, gvel = h.get_state(0)
    gphi, gq = h.densities(0)
    assert fluct_err(gom, st.omega) < 1e-10
    assert rel_err(gphi, st.phi) < 1e-10
    assert rel_err(gq, st.q) < 1e-12
    assert rel_err(gvel, st.vel) < 1e-9
    assert np.abs(gpop - st.pop).max() < 1e-13
    h.close()


def test_exact_step_fp64_converges_with_the_oracle():
    ny, nx, ns = 32, 64, 8
    r = P.RunParams(nx=nx, ny=ny, ns=ns, precision=P.PLAIN_FP64, f_a=0.5, phi_p=0.2, f0=10.0)
    omega, pop, vel = _random_state(ny, nx, 41, 0.002)
    h = P.EpdLb([r])
    h.set_state(0, omega, pop, vel)
    h.set_inversion(80, 1e-8)
    h.step(2)
    h.sync()
    st, stats = _oracle_exact(r, omega, pop, vel, 80, 1e-8, nsteps=2)
    s = h.inversion_stats(0)
    assert 0 < s["iterations"] == int(stats[1, 0]) and s["residual"] < 1e-8
    assert abs(s["residual"] - stats[1, 2]) <= 1e-6 * stats[1, 2]
    gom, _, gvel = h.get_state(0)
    gphi, _ = h.densities(0)
    assert fluct_err(gom, st.omega) < 1e-9
    assert rel_err(gphi, st.phi) < 1e-10
    assert rel_err(gvel, st.vel) < 1e-8
    h.close()


@pytest.mark.parametrize("ny,nx,ns", [(64, 64, 16), (64, 128, 10), (32, 64, 8), (64, 1024, 8), (60, 96, 12)])
def test_exact_step_mixed_cluster_converges(ny, nx, ns):
    # MIXED_FP32 with the differential solves (cluster-resident on 64 x 64
    # and 128 x 64; streaming generic, radix-8 and mixed-radix on the
    # others): every density of the step is
    # a difference from the solve at the starting guess, so the mismatch
    # reaches the paper's 1e-8 although FP32 densities differ from FP64 by
    # ~3e-7.  omega~ inverts the FP32 density map: its distance from the FP64
    # inverse is that density error times the inverse correlator, whose
    # largest eigenvalue (the inverse of the short-wavelength polymer
    # response, ~0.03 here) amplifies it about 30-fold
    r = P.RunParams(nx=nx, ny=ny, ns=ns, precision=P.MIXED_FP32, f_a=0.5, phi_p=0.2, f0=2.0)
    omega, pop, vel = _random_state(ny, nx, 51, 0.002)
    h = P.EpdLb([r])
    assert h.tiles(0)["differential"]
    h.set_state(0, omega, pop, vel)
    h.set_inversion(80, 1e-8)
    h.step(1)
    h.sync()
    st, stats = _oracle_exact(r, omega, pop, vel, 80, 1e-8)
    s = h.inversion_stats(0)
    assert s["residual"] < 1e-8 and abs(s["iterations"] - stats[0, 0]) <= 3
    assert abs(s["residual0"] - stats[0, 1]) <= 1e-4 * stats[0, 1]
    gom, _, gvel = h.get_state(0)
    gphi, _ = h.densities(0)
    assert fluct_err(gom, st.omega) < 1e-5
    assert rel_err(gphi, st.phi) < 2e-6
    h.close()


@pytest.mark.parametrize("prec", [P.PLAIN_FP64, P.MIXED_FP32])
def test_exact_step_without_iterations_is_the_truncated_step(prec):
    # a tolerance above the starting residual: no iteration, and the state
    # is bitwise that of the graph-captured truncated step
    r = W.with_(W.plain_small(), nx=64, ny=64, ns=16, precision=prec, f0=2.0, seed=9)
    a, b = P.EpdLb([r]), P.EpdLb([r])
    b.set_inversion(10, 1.0)
    a.step(2)
    b.step(2)
    assert b.inversion_stats(0)["iterations"] == 0
    for x, y in zip(a.get_state(0), b.get_state(0)):
        assert np.array_equal(x, y)
    assert np.array_equal(a.densities(0)[0], b.densities(0)[0])
    a.close()
    b.close()


def test_exact_step_batch_iterates_each_run_to_its_tolerance():
    ny, nx, ns = 32, 32, 8
    runs = [P.RunParams(nx=nx, ny=ny, ns=ns, precision=P.PLAIN_FP64, f_a=0.5, phi_p=0.2, f0=10.0, seed=3 + k)
            for k in range(3)]
    states = [_random_state(ny, nx, 61 + 10 * k, a) for k, a in enumerate((0.0005, 0.002, 0.008))]
    h = P.EpdLb(runs)
    for k, (om, pop, vel) in enumerate(states):
        h.set_state(k, om, pop, vel)
    h.set_inversion(80, 1e-8)
    h.step(1)
    h.sync()
    iters = []
    for k, (om, pop, vel) in enumerate(states):
        st, stats = _oracle_exact(runs[k], om, pop, vel, 80, 1e-8)
        s = h.inversion_stats(k)
        assert s["iterations"] == int(stats[0, 0]) and s["residual"] < 1e-8
        gom, _, _ = h.get_state(k)
        assert fluct_err(gom, st.omega) < 1e-9
        iters.append(s["iterations"])
    assert len(set(iters)) > 1  # the runs stopped at different iterations
    h.close()


def test_exact_step_errors():
    # not converged within max_iter: the step completes, then ENOTCONV
    r = P.RunParams(nx=32, ny=32, ns=8, precision=P.PLAIN_FP64, f_a=0.5, phi_p=0.2, f0=10.0)
    omega, pop, vel = _random_state(32, 32, 71, 0.02)
    h = P.EpdLb([r])
    h.set_state(0, omega, pop, vel)
    h.set_inversion(1, 1e-30)
    with pytest.raises(P.EpdLbError) as e:
        h.step(1)
    assert e.value.code == -7
    assert h.inversion_stats(0)["iterations"] == 1
    with pytest.raises(P.EpdLbError):
        h.set_inversion(-1, 1e-8)
    with pytest.raises(P.EpdLbError):
        h.set_inversion(5, float("nan"))
    h.close()


def test_exact_step_at_the_benchmark_size():
    # the benchmark batch's strongest-shear run (256 x 512, N_s = 64, MIXED,
    # cluster-resident differential solves) from the seeded quench: two
    # truncated steps, then an exact step with two CG iterations, against the
    # FP64 oracle doing the same
    r = W.channel_256x512(P.MIXED_FP32)[3]
    h = P.EpdLb([r])
    h.step(2)
    h.set_inversion(2, 0.0)
    h.step(1)
    h.sync()
    p = oracle_params(r)
    st = O.initial_state(p)
    O.step(p, st, 2)
    stats = O.step_exact(p, st, 1, max_iter=2, tol=0.0)
    s = h.inversion_stats(0)
    assert s["iterations"] == 2 == int(stats[0, 0])
    assert abs(s["residual0"] - stats[0, 1]) <= 2e-3 * stats[0, 1]
    gom, _, gvel = h.get_state(0)
    gphi, _ = h.densities(0)
    # the absolute bound of the 64 x 64 case above (1e-5 of a 0.05 spread):
    # FP32 density error times the inverse correlator, independent of how
    # large the fluctuations of omega are (here ~1e-3)
    assert np.abs(gom - st.omega).max() < 5e-7
    assert rel_err(gphi, st.phi) < 2e-6
    h.close()
