"""GPU coupled EPD/LB step against the FP64 oracle: initial state, single
steps from arbitrary states, multi-step runs, the full-size batch that the
benchmark times, invariants, checkpoints and error handling."""
import numpy as np
import pytest

import oracle as O
import paper_1804_02883_gb300 as P
from paper_1804_02883_gb300 import workloads as W
from helpers import fluct_err, oracle_params, rel_err, vel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build(oracle_lib):
    P.lib()


def oracle_state_from(r, omega, pop, vel):
    p = oracle_params(r)
    phi, q = O.solve(p, omega)
    return p, O.State(omega.copy(), pop.copy(), vel.copy(), phi, q, np.zeros((2, r.ny, r.nx)))


@pytest.mark.parametrize("prec", [P.PLAIN_FP64, P.MIXED_FP32])
def test_initial_state_matches_oracle(prec):
    r = W.with_(W.plain_small(), nx=32, ny=16, ns=8, precision=prec, f0=200.0, seed=77)
    h = P.EpdLb([r])
    om, pop, vel = h.get_state(0)
    oom, opop, ovel = O.init(oracle_params(r))
    assert np.array_equal(om, oom)  # same counter-based generator, same FP64 ops
    tol = 1e-15 if prec == P.PLAIN_FP64 else 1e-7
    assert np.abs(pop - opop).max() < tol
    assert np.abs(vel - ovel).max() < tol * max(1e-30, np.abs(ovel).max()) + 1e-20
    phi, q = h.densities(0)
    ophi, oq = O.solve(oracle_params(r), oom)
    assert rel_err(phi, ophi) < (1e-10 if prec == P.PLAIN_FP64 else 2e-5)
    h.close()


@pytest.mark.parametrize("ny,nx,ns", [(16, 32, 8), (64, 32, 12), (8, 128, 6)])
def test_single_step_from_random_state_fp64(ny, nx, ns):
    r = P.RunParams(nx=nx, ny=ny, ns=ns, precision=P.PLAIN_FP64, f_a=0.5, phi_p=0.2, f0=10.0)
    omega = W.random_omega(ny, nx, seed=5, amp=0.05)
    pop = W.random_populations(ny, nx, seed=6)
    vel = W.random_velocity(ny, nx, seed=7, amp=0.02)
    h = P.EpdLb([r])
    h.set_state(0, omega, pop, vel)
    h.step(1)
    h.sync()
    p, st = oracle_state_from(r, omega, pop, vel)
    O.step(p, st)
    gom, gpop, gvel = h.get_state(0)
    gphi, gq = h.densities(0)
    assert fluct_err(gom, st.omega) < 1e-10
    assert rel_err(gphi, st.phi) < 1e-10
    assert rel_err(gq, st.q) < 1e-12
    assert rel_err(gvel, st.vel) < 1e-10
    assert np.abs(gpop - st.pop).max() < 1e-14
    h.close()


def test_single_step_mixed_precision():
    ny, nx, ns = 32, 64, 16
    r = P.RunParams(nx=nx, ny=ny, ns=ns, precision=P.MIXED_FP32, f_a=0.5, phi_p=0.2, f0=10.0)
    omega = W.random_omega(ny, nx, seed=15, amp=0.05)
    pop = W.random_populations(ny, nx, seed=16)
    vel = W.random_velocity(ny, nx, seed=17, amp=0.02)
    h = P.EpdLb([r])
    # 64 x 32 takes the generic streaming solve; its second solve is the
    # change from the first (differential), so the force that dPhi^D ~ 2e-3
    # drives keeps FP32 precision relative to dPhi^D itself
    t = h.tiles(0)
    assert t["path"] == 0 and t["differential"]
    h.set_state(0, omega, pop, vel)
    h.step(1)
    p, st = oracle_state_from(r, omega, pop, vel)
    O.step(p, st)
    gom, gpop, gvel = h.get_state(0)
    gphi, _ = h.densities(0)
    assert fluct_err(gom, st.omega) < 2e-6
    assert rel_err(gphi, st.phi) < 2e-6
    assert rel_err(gvel, st.vel) < 1e-5
    assert np.abs(gpop - st.pop).max() < 1e-7
    h.close()


@pytest.mark.parametrize("nx,ny,ns,f_a", [(150, 150, 16, 0.5), (150, 150, 17, 0.882), (96, 60, 12, 0.3)])
def test_single_step_mixed_mixed_radix_grid(nx, ny, ns, f_a):
    # the paper's 150 x 150 grid (and another 2^a 3^b 5^c one): mixed-radix
    # streaming passes with the differential second solve
    r = P.RunParams(nx=nx, ny=ny, ns=ns, precision=P.MIXED_FP32, f_a=f_a, phi_p=0.2, f0=0.5)
    omega = W.random_omega(ny, nx, seed=51, amp=0.05)
    pop = W.random_populations(ny, nx, seed=52)
    vel = W.random_velocity(ny, nx, seed=53, amp=0.02)
    h = P.EpdLb([r])
    t = h.tiles(0)
    assert t["path"] == 0 and t["differential"]
    h.set_state(0, omega, pop, vel)
    h.step(1)
    p, st = oracle_state_from(r, omega, pop, vel)
    O.step(p, st)
    gom, gpop, gvel = h.get_state(0)
    gphi, gq = h.densities(0)
    assert rel_err(gphi, st.phi) < 2e-6
    assert rel_err(gq, st.q) < 2e-6
    assert fluct_err(gom, st.omega) < 2e-6
    assert rel_err(gvel, st.vel) < 1e-5
    assert np.abs(gpop - st.pop).max() < 1e-7
    h.close()


@pytest.mark.parametrize("ny,nx,ns", [(64, 64, 16), (64, 128, 10), (128, 64, 20)])
def test_single_step_mixed_differential_solve(ny, nx, ns):
    # cluster-solve grids: the second solve is carried as the change from the
    # first, so dPhi^D and the force it drives keep FP32 precision relative
    # to themselves (1e-7 of dPhi^D, not of Phi)
    r = P.RunParams(nx=nx, ny=ny, ns=ns, precision=P.MIXED_FP32, f_a=0.3, phi_p=0.2, f0=2.0)
    omega = W.random_omega(ny, nx, seed=31, amp=0.05)
    pop = W.random_populations(ny, nx, seed=32)
    vel = W.random_velocity(ny, nx, seed=33, amp=0.02)
    h = P.EpdLb([r])
    h.set_state(0, omega, pop, vel)
    h.step(1)
    p, st = oracle_state_from(r, omega, pop, vel)
    O.step(p, st)
    gom, gpop, gvel = h.get_state(0)
    gphi, gq = h.densities(0)
    assert rel_err(gphi, st.phi) < 2e-6
    assert rel_err(gq, st.q) < 2e-6
    assert fluct_err(gom, st.omega) < 2e-6
    assert rel_err(gvel, st.vel) < 1e-5
    assert np.abs(gpop - st.pop).max() < 1e-7
    h.close()


@pytest.mark.parametrize("ny,nx,ns,f_a,f0", [(64, 1024, 8, 0.5, 10.0), (128, 1024, 16, 0.3, 2.0)])
def test_single_step_mixed_streaming_radix8(ny, nx, ns, f_a, f0):
    # no cluster shape: radix-8 streaming passes with the full history, the
    # second solve as the change from the first against that history
    r = P.RunParams(nx=nx, ny=ny, ns=ns, precision=P.MIXED_FP32, f_a=f_a, phi_p=0.2, f0=f0)
    omega = W.random_omega(ny, nx, seed=41, amp=0.05)
    pop = W.random_populations(ny, nx, seed=42)
    vel = W.random_velocity(ny, nx, seed=43, amp=0.02)
    h = P.EpdLb([r])
    t = h.tiles(0)
    assert t["path"] == 1 and t["differential"]
    h.set_state(0, omega, pop, vel)
    h.step(1)
    p, st = oracle_state_from(r, omega, pop, vel)
    O.step(p, st)
    gom, gpop, gvel = h.get_state(0)
    gphi, gq = h.densities(0)
    assert rel_err(gphi, st.phi) < 2e-6
    assert rel_err(gq, st.q) < 2e-6
    assert fluct_err(gom, st.omega) < 2e-6
    assert rel_err(gvel, st.vel) < 1e-5
    assert np.abs(gpop - st.pop).max() < 1e-7
    h.close()


def test_mixed_tracks_fp64_over_100_steps():
    # 64 x 64, N_s = 32 from the seeded quench: MIXED and PLAIN_FP64 side by
    # side; the remaining velocity difference comes from the FP32 resolution
    # of the density fluctuations (~1e-7 of Phi against fluctuations ~1e-4)
    r64 = W.plain_small()
    a = P.EpdLb([r64])
    b = P.EpdLb([W.with_(r64, precision=P.MIXED_FP32)])
    a.step(100)
    b.step(100)
    pa, qa = a.densities(0)
    pb, qb = b.densities(0)
    assert rel_err(pb, pa) < 1e-6
    assert rel_err(qb, qa) < 1e-6
    assert rel_err(b.velocity(0), a.velocity(0)) < 5e-3
    a.close()
    b.close()


def test_multi_step_from_init_fp64():
    # the small FP64 configuration (64 x 64, N_s = 32, f0 = 1e-6) over its
    # full 200 coupled steps, compared every 20 steps
    r = W.plain_small()
    h = P.EpdLb([r])
    p = oracle_params(r)
    st = O.initial_state(p)
    for k in range(10):
        h.step(20)
        O.step(p, st, 20)
        gphi, gq = h.densities(0)
        gom, gpop, gvel = h.get_state(0)
        assert rel_err(gphi, st.phi) < 1e-10, k
        assert fluct_err(gphi[0] + gphi[1], st.phi[0] + st.phi[1]) < 1e-8, k
        assert fluct_err(gom, st.omega) < 1e-9, k
        assert vel_err(gvel, st.vel, 1e-9) < 1, k
    h.close()


def test_mixed_tracks_the_fp64_oracle_over_1000_steps():
    # The reduced-precision bar: the mixed-precision path (FP32 propagators,
    # LB and EPD transforms; FP64 fields, contour sums, Q, masses) against the
    # FP64 oracle after 1000 coupled steps of the 64 x 64, N_s = 32 quench,
    # densities within 1e-5 relative.  The velocity follows the density
    # fluctuations (~1e-4 here), which FP32 resolves to ~3e-4 of themselves,
    # so it is held to 2e-2 of max |u|.
    r = W.with_(W.plain_small(), precision=P.MIXED_FP32)
    h = P.EpdLb([r])
    p = oracle_params(r)
    st = O.initial_state(p)
    for k in range(4):
        h.step(250)
        O.step(p, st, 250)
        gphi, gq = h.densities(0)
        assert rel_err(gphi, st.phi) < 1e-5, k
        assert rel_err(gq, st.q) < 1e-5, k
    gom, _, gvel = h.get_state(0)
    assert fluct_err(gphi[0] + gphi[1], st.phi[0] + st.phi[1]) < 1e-2
    assert rel_err(gvel, st.vel) < 2e-2
    h.close()


@pytest.mark.parametrize("nx,ny,ns", [(96, 60, 12), (1024, 64, 16)])
def test_mixed_streaming_tracks_the_fp64_oracle(nx, ny, ns):
    # the streaming paths (mixed-radix on 96 x 60, whose oracle transforms are
    # the DFT by definition; radix-8 on 1024 x 64) over 100 coupled steps of
    # a quench in shear, compared with the FP64 oracle every 25 steps
    r = P.RunParams(nx=nx, ny=ny, ns=ns, precision=P.MIXED_FP32, f_a=0.5, phi_p=0.2, f0=0.5, noise_amp=1e-3, seed=8)
    h = P.EpdLb([r])
    p = oracle_params(r)
    st = O.initial_state(p)
    for k in range(4):
        h.step(25)
        O.step(p, st, 25)
        gphi, gq = h.densities(0)
        e_phi, e_q, e_v = rel_err(gphi, st.phi), rel_err(gq, st.q), rel_err(h.velocity(0), st.vel)
        assert e_phi < 1e-5 and e_q < 1e-5 and e_v < 1e-4, (k, e_phi, e_q, e_v)
    h.close()


def test_full_size_batch_first_run_matches_oracle():
    # The launch configuration the benchmark times: four 256 x 512 runs,
    # N_s = 64, mixed precision.  One step from a random state of run 0
    # against one oracle step; the other runs by invariants.
    runs = W.channel_256x512(P.MIXED_FP32)
    h = P.EpdLb(runs)
    r = runs[2]
    omega = W.random_omega(r.ny, r.nx, seed=21, amp=0.02)
    pop = W.random_populations(r.ny, r.nx, seed=22, amp=1e-4)
    vel = W.random_velocity(r.ny, r.nx, seed=23, amp=1e-3)
    h.set_state(2, omega, pop, vel)
    h.step(1)
    p, st = oracle_state_from(r, omega, pop, vel)
    O.step(p, st)
    gphi, gq = h.densities(2)
    gom, gpop, gvel = h.get_state(2)
    assert rel_err(gphi, st.phi) < 2e-6
    assert fluct_err(gom, st.omega) < 2e-6
    # the second solve is the change from the first (differential solve), so
    # the force keeps FP32 precision relative to dPhi^D (measured 2.5e-7)
    assert rel_err(gvel, st.vel) < 1e-5
    for k in (0, 1, 3):
        ob = h.observables(k)
        assert abs((ob["mean_phi_a"] + ob["mean_phi_b"]) / runs[k].phi_p - 1) < 1e-6
        assert abs(ob["lb_mass"] - 1) < 1e-6
    h.close()


def test_full_size_batch_every_run_matches_oracle():
    # the benchmark's launch configuration (four 256 x 512 runs, N_s = 64,
    # the phased differential chain schedule): one step from a random state
    # of every run against one oracle step of that run
    runs = W.channel_256x512(P.MIXED_FP32)
    h = P.EpdLb(runs)
    states = []
    for k, r in enumerate(runs):
        st = (W.random_omega(r.ny, r.nx, seed=60 + k, amp=0.02), W.random_populations(r.ny, r.nx, seed=70 + k, amp=1e-4),
              W.random_velocity(r.ny, r.nx, seed=80 + k, amp=1e-3))
        h.set_state(k, *st)
        states.append(st)
    h.step(1)
    for k, r in enumerate(runs):
        p, st = oracle_state_from(r, *states[k])
        O.step(p, st)
        gphi, gq = h.densities(k)
        gom, gpop, gvel = h.get_state(k)
        assert rel_err(gphi, st.phi) < 2e-6, k
        assert rel_err(gq, st.q) < 2e-6, k
        assert fluct_err(gom, st.omega) < 2e-6, k
        assert rel_err(gvel, st.vel) < 1e-5, k
        assert np.abs(gpop - st.pop).max() < 1e-7, k
    h.close()


def test_vesicle_grid_step_matches_oracle():
    # the 1024 x 2048 vesicle configuration's grid and parameters (radix-8
    # streaming passes, differential second solve) with a short chain,
    # N_s = 16, so that the oracle step takes seconds; one step from a
    # random state against the oracle
    r = W.with_(W.vesicle_1024x2048(P.MIXED_FP32), ns=16)
    h = P.EpdLb([r])
    assert h.tiles(0)["path"] == 1 and h.tiles(0)["differential"]
    omega = W.random_omega(r.ny, r.nx, seed=91, amp=0.02)
    pop = W.random_populations(r.ny, r.nx, seed=92, amp=1e-4)
    vel = W.random_velocity(r.ny, r.nx, seed=93, amp=1e-3)
    h.set_state(0, omega, pop, vel)
    h.step(1)
    p, st = oracle_state_from(r, omega, pop, vel)
    O.step(p, st)
    gphi, gq = h.densities(0)
    gom, gpop, gvel = h.get_state(0)
    assert rel_err(gphi, st.phi) < 2e-6
    assert rel_err(gq, st.q) < 2e-6
    assert fluct_err(gom, st.omega) < 2e-6
    assert rel_err(gvel, st.vel) < 1e-5
    assert np.abs(gpop - st.pop).max() < 1e-7
    h.close()


def test_vesicle_configuration_invariants():
    # the full 1024 x 2048, N_s = 128 configuration the benchmark times:
    # properties that hold at any size after three steps from the seeded
    # quench -- each species' mass (Eqs. (2), (5)), the LB mass, Q > 0
    r = W.vesicle_1024x2048(P.MIXED_FP32)
    h = P.EpdLb([r])
    h.step(3)
    h.sync()
    ob = h.observables(0)
    na = round(r.f_a * r.ns)
    assert abs(ob["mean_phi_a"] / (r.phi_p * na / r.ns) - 1) < 1e-6
    assert abs(ob["mean_phi_b"] / (r.phi_p * (r.ns - na) / r.ns) - 1) < 1e-6
    assert abs(ob["mean_phi_s"] / (1 - r.phi_p) - 1) < 1e-6
    assert abs(ob["lb_mass"] - 1) < 1e-6
    assert ob["q_p"] > 0 and ob["q_s"] > 0
    h.close()


def test_batch_equals_single_runs():
    runs = [W.with_(W.plain_small(), nx=32, ny=32, ns=8, seed=s, f0=f) for s, f in ((1, 0.0), (2, 20.0), (3, 50.0))]
    hb = P.EpdLb(runs)
    hb.step(3)
    for k, r in enumerate(runs):
        hs = P.EpdLb([r])
        hs.step(3)
        a, _ = hb.densities(k)
        b, _ = hs.densities(0)
        assert np.array_equal(a, b)
        hs.close()
    hb.close()


def test_phased_chain_schedule_equals_single_runs():
    # four 256 x 512 runs are 8 chains of 16-CTA clusters; where only 7 fit at
    # one CTA per SM the chains take turns over 8 launches, resuming from the
    # FP32 states they stored, so the batch still equals each run stepped
    # alone (one launch of 2 chains) bit for bit, in both solves
    runs = W.channel_256x512(P.MIXED_FP32)
    hb = P.EpdLb(runs)
    t = hb.tiles(0)
    assert t["path"] == 2 and t["differential"] and t["chain_launches"] in (1, 2 * len(runs))
    hb.step(2)
    for k, r in enumerate(runs):
        hs = P.EpdLb([r])
        assert hs.tiles(0)["chain_launches"] == 1
        hs.step(2)
        assert np.array_equal(hb.densities(k)[0], hs.densities(0)[0])
        assert np.array_equal(hb.velocity(k), hs.velocity(0))
        hs.close()
    hb.close()


def test_dependent_chain_launches_do_not_change_results():
    # the phased schedule's launches after the first are programmatic
    # dependents of the one before; EPD_LB_CHAIN_PDL=0 (read when the library
    # loads) launches them plainly.  Both give the same bits.
    import json
    import os
    import subprocess
    import sys

    code = (
        "import json, numpy as np\n"
        "import paper_1804_02883_gb300 as P\n"
        "from paper_1804_02883_gb300 import workloads as W\n"
        "h = P.EpdLb(W.channel_256x512(P.MIXED_FP32))\n"
        "assert h.tiles(0)['chain_launches'] in (1, 8)\n"
        "h.step(3)\n"
        "phi, q = h.densities(1)\n"
        "print(json.dumps({'launches': h.tiles(0)['chain_launches'], 'phi': float(np.abs(phi).sum()), "
        "'first': phi.ravel()[:64].tolist(), 'q': q.tolist(), 'u': h.velocity(1).ravel()[:64].tolist()}))\n"
        "h.close()\n")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = []
    for pdl in ("1", "0"):
        env = dict(os.environ, EPD_LB_CHAIN_PDL=pdl)
        r = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        out.append(json.loads(r.stdout.strip().splitlines()[-1]))
    assert out[0] == out[1]


def test_uneven_batch_groups_match_single_runs():
    runs = [P.RunParams(nx=32, ny=16, ns=8, precision=P.MIXED_FP32, seed=1),
            P.RunParams(nx=16, ny=32, ns=12, precision=P.MIXED_FP32, seed=2),
            P.RunParams(nx=32, ny=16, ns=8, precision=P.MIXED_FP32, seed=3, f0=100.0)]
    hb = P.EpdLb(runs)
    hb.step(4)
    for k, r in enumerate(runs):
        hs = P.EpdLb([r])
        hs.step(4)
        assert np.array_equal(hb.densities(k)[0], hs.densities(0)[0])
        hs.close()
    hb.close()


def test_invariants_over_many_steps_mixed():
    r = W.with_(W.plain_small(), precision=P.MIXED_FP32, f0=10.0)
    h = P.EpdLb([r])
    h.step(200)
    h.sync()
    ob = h.observables(0)
    assert abs((ob["mean_phi_a"] + ob["mean_phi_b"]) / r.phi_p - 1) < 1e-6
    assert abs(ob["mean_phi_s"] / (1 - r.phi_p) - 1) < 1e-12
    assert abs(ob["lb_mass"] - 1) < 1e-6
    assert np.isfinite(ob["sigma"]) and ob["q_p"] > 0
    h.close()


def test_checkpoint_resume_is_bitwise():
    r = W.with_(W.plain_small(), nx=32, ny=32, ns=8, f0=50.0)
    a = P.EpdLb([r])
    a.step(3)
    blob = a.save()
    a.step(4)
    b = P.EpdLb([r])
    b.load(blob)
    b.step(4)
    assert np.array_equal(a.densities(0)[0], b.densities(0)[0])
    assert np.array_equal(a.velocity(0), b.velocity(0))
    a.close()
    b.close()


def test_supersonic_poiseuille_refused():
    r = W.with_(W.plain_small(), f0=1e9)
    with pytest.raises(P.EpdLbError) as ei:
        P.EpdLb([r])
    assert ei.value.code == -5


def test_decoupled_run_keeps_fluid_at_rest():
    r = W.with_(W.plain_small(), nx=32, ny=32, ns=8, f0=0.0, inv_beta_v=0.0, noise_amp=1e-2)
    h = P.EpdLb([r])
    h.step(5)
    assert np.all(h.velocity(0) == 0)
    h.close()


def test_async_host_buffer_calls_match_synchronous_ones():
    # epd_lb_set_omega_async / epd_lb_densities_async enqueue the same copies
    # as epd_lb_set_state / epd_lb_densities without a synchronisation
    import torch

    r = W.with_(W.plain_small(), precision=P.MIXED_FP32, nx=64, ny=64)
    a, b = P.EpdLb([r]), P.EpdLb([r])
    om = W.random_omega(r.ny, r.nx, seed=71, amp=0.05)
    host_om = torch.from_numpy(om.ravel().copy()).pin_memory()
    host_phi = torch.empty(3 * r.nx * r.ny, dtype=torch.float64).pin_memory()
    host_q = torch.empty(2, dtype=torch.float64).pin_memory()
    a.set_state(0, om, None, None)
    a.step(2)
    phi_a, q_a = a.densities(0)
    b.set_omega_async(0, host_om.data_ptr())
    b.step(2)
    b.densities_async(0, host_phi.data_ptr(), host_q.data_ptr())
    b.sync()
    assert np.array_equal(host_phi.numpy().reshape(3, r.ny, r.nx), phi_a)
    assert np.array_equal(host_q.numpy(), q_a)
    a.close()
    b.close()
