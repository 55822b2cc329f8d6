"""GPU path on grids whose sides are not powers of two (the paper's own
150 x 150 grid and other 2^a 3^b 5^c sides): mixed-radix (2, 3, 4, 5)
shared-memory transforms in the streaming propagator and EPD passes, LB with
general periodic indexing.  Against the FP64 oracle (whose transforms are
the DFT by definition on such axes): solves, the initial state, single and
exact steps, particles."""
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


@pytest.mark.parametrize("prec", [P.PLAIN_FP64, P.MIXED_FP32])
@pytest.mark.parametrize("nx,ny,ns", [(30, 20, 8), (24, 40, 10), (96, 60, 12), (150, 150, 16)])
def test_solve_matches_oracle(prec, nx, ny, ns):
    r = P.RunParams(nx=nx, ny=ny, ns=ns, precision=prec, f_a=0.5, phi_p=0.2, f0=0.0)
    omega = W.random_omega(ny, nx, seed=nx + ny, amp=0.1)
    h = P.EpdLb([r])
    assert h.tiles(0)["path"] == 0  # the radix-2-family passes with mixed-radix transforms
    phi, q = h.solve(0, omega)
    ophi, oq = O.solve(oracle_params(r), omega)
    tol = 1e-12 if prec == P.PLAIN_FP64 else 2e-6
    assert rel_err(phi, ophi) < tol
    assert rel_err(q, oq) < tol
    h.close()


def test_initial_state_on_the_paper_grid():
    r = P.RunParams(nx=150, ny=150, ns=16, precision=P.PLAIN_FP64, f_a=0.5, phi_p=0.2, f0=1e-4, seed=11)
    h = P.EpdLb([r])
    om, pop, vel = h.get_state(0)
    oom, opop, ovel = O.init(oracle_params(r))
    assert np.array_equal(om, oom)
    assert np.abs(pop - opop).max() < 1e-15
    phi, _ = h.densities(0)
    ophi, _ = O.solve(oracle_params(r), oom)
    assert rel_err(phi, ophi) < 1e-12
    h.close()


@pytest.mark.parametrize("nx,ny,ns", [(30, 20, 8), (150, 150, 16)])
def test_single_step_fp64(nx, ny, ns):
    # the body force kept below the Mach-number pre-flight on the 150-wide channel
    r = P.RunParams(nx=nx, ny=ny, ns=ns, precision=P.PLAIN_FP64, f_a=0.5, phi_p=0.2, f0=10.0 if ny < 100 else 0.5)
    omega = W.random_omega(ny, nx, seed=5, amp=0.05)
    pop = W.random_populations(ny, nx, seed=6)
    vel = W.random_velocity(ny, nx, seed=7, amp=0.02)
    h = P.EpdLb([r])
    h.set_state(0, omega, pop, vel)
    h.step(1)
    h.sync()
    p = oracle_params(r)
    phi, q = O.solve(p, omega)
    st = O.State(omega.copy(), pop.copy(), vel.copy(), phi, q, np.zeros((2, ny, nx)))
    O.step(p, st)
    gom, gpop, gvel = h.get_state(0)
    gphi, gq = h.densities(0)
    assert fluct_err(gom, st.omega) < 1e-10
    assert rel_err(gphi, st.phi) < 1e-10
    assert rel_err(gq, st.q) < 1e-12
    assert rel_err(gvel, st.vel) < 1e-9
    assert np.abs(gpop - st.pop).max() < 1e-13
    h.close()


@pytest.mark.parametrize("prec,nx,ny", [(P.PLAIN_FP64, 30, 20), (P.MIXED_FP32, 30, 20), (P.PLAIN_FP64, 32, 32)])
def test_odd_contour_count_step(prec, nx, ny):
    # N_s = N = 17 with q_A = 0.882 (15 A intervals), the paper's own chain
    r = P.RunParams(nx=nx, ny=ny, ns=17, precision=prec, f_a=0.882, phi_p=0.1, f0=10.0)
    omega = W.random_omega(ny, nx, seed=25, amp=0.05)
    pop = W.random_populations(ny, nx, seed=26)
    vel = W.random_velocity(ny, nx, seed=27, amp=0.02)
    h = P.EpdLb([r])
    h.set_state(0, omega, pop, vel)
    h.step(1)
    h.sync()
    p = oracle_params(r)
    phi, q = O.solve(p, omega)
    st = O.State(omega.copy(), pop.copy(), vel.copy(), phi, q, np.zeros((2, ny, nx)))
    O.step(p, st)
    gom, _, _ = h.get_state(0)
    gphi, gq = h.densities(0)
    tol = 1e-10 if prec == P.PLAIN_FP64 else 2e-6
    assert fluct_err(gom, st.omega) < tol
    assert rel_err(gphi, st.phi) < tol
    assert rel_err(gq, st.q) < tol
    h.close()


def test_steps_mixed_precision_track_fp64():
    # MIXED against PLAIN on a 96 x 60 grid over 20 steps from the seeded quench
    base = P.RunParams(nx=96, ny=60, ns=12, precision=P.PLAIN_FP64, f_a=0.5, phi_p=0.2, f0=2.0, noise_amp=1e-3, seed=4)
    a, b = P.EpdLb([base]), P.EpdLb([W.with_(base, precision=P.MIXED_FP32)])
    a.step(20)
    b.step(20)
    pa, _ = a.densities(0)
    pb, _ = b.densities(0)
    assert rel_err(pb, pa) < 1e-6, rel_err(pb, pa)
    assert fluct_err(pb, pa) < 5e-3, fluct_err(pb, pa)
    a.close()
    b.close()


def test_exact_step_on_a_mixed_radix_grid():
    r = P.RunParams(nx=30, ny=20, ns=8, precision=P.PLAIN_FP64, f_a=0.5, phi_p=0.2, f0=10.0)
    omega = W.random_omega(20, 30, seed=15, amp=0.05)
    pop = W.random_populations(20, 30, seed=16)
    vel = W.random_velocity(20, 30, seed=17, amp=0.02)
    h = P.EpdLb([r])
    h.set_state(0, omega, pop, vel)
    h.set_inversion(3, 0.0)
    h.step(1)
    h.sync()
    p = oracle_params(r)
    phi, q = O.solve(p, omega)
    st = O.State(omega.copy(), pop.copy(), vel.copy(), phi, q, np.zeros((2, 20, 30)))
    O.step_exact(p, st, 1, max_iter=3, tol=0.0)
    gom, _, _ = h.get_state(0)
    gphi, _ = h.densities(0)
    assert fluct_err(gom, st.omega) < 1e-10
    assert rel_err(gphi, st.phi) < 1e-10
    h.close()
