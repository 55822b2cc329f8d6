"""Pins of the oracle's coupled step (App. C) and initial state (Sec. 3-4):
invariants that hold exactly for any state (mass of every species, LB mass,
LB momentum since the force has zero mean), special cases that reduce the
step to a known answer, and the splitmix64 generator's published outputs."""
import os

import numpy as np

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])


def test_splitmix64_published_outputs(oracle_lib):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "splitmix64.txt")) if not l.startswith("#")]
    for k, out in rows:
        assert O.splitmix64(int(k) * 0x9E3779B97F4A7C15) == int(out, 16)


def test_noise_uniform(oracle_lib):
    vals = np.array([O.noise(11, c) for c in range(20000)])
    assert vals.min() >= -1 and vals.max() < 1
    hist, _ = np.histogram(vals, bins=10, range=(-1, 1))
    assert np.all(np.abs(hist - 2000) < 5 * np.sqrt(2000))


def test_initial_state(oracle_lib):
    p = O.Params(nx=8, ny=16, f0=5.0, noise_amp=1e-3, seed=42)
    omega, pop, vel = O.init(p)
    assert np.abs(omega).max() <= 1e-3
    assert omega[1, 3, 5] == 1e-3 * O.noise(42, (1 * p.ny + 3) * p.nx + 5)
    assert np.allclose(pop.sum(0), 1.0, rtol=0, atol=1e-15)
    want = np.array([O.discrete_profile(p, y) for y in range(p.ny)])
    assert np.all(vel[0] == want[:, None]) and np.all(vel[1] == 0)
    # the first collision sees u = v(y): j = v - f_P/2
    fP = np.array([O.poiseuille_force(p, y) for y in range(p.ny)])
    jx = (CX[:, None, None] * pop).sum(0)
    assert np.abs(jx + fP[:, None] / 2 - vel[0]).max() < 1e-16


def test_step_invariants(oracle_lib):
    p = O.Params(nx=16, ny=32, ns=8, phi_p=0.2, f0=20.0, noise_amp=5e-2, seed=3)
    st = O.initial_state(p)
    m0 = st.pop.sum()
    jx0 = (CX[:, None, None] * st.pop).sum()
    jy0 = (CY[:, None, None] * st.pop).sum()
    for _ in range(3):
        O.step(p, st)
        assert abs(st.phi[0].mean() + st.phi[1].mean() - p.phi_p) < 1e-14
        assert abs(st.phi[2].mean() - (1 - p.phi_p)) < 1e-14
        assert abs(st.force[0].sum()) < 1e-12 * np.abs(st.force).sum()
    assert abs(st.pop.sum() - m0) < 1e-12
    assert abs((CX[:, None, None] * st.pop).sum() - jx0) < 1e-14
    assert abs((CY[:, None, None] * st.pop).sum() - jy0) < 1e-14
    assert np.abs(st.force).max() > 0


def test_homogeneous_state_is_stationary(oracle_lib):
    p = O.Params(nx=8, ny=8, ns=6, f0=0.0, noise_amp=0.0)
    st = O.initial_state(p)
    st.omega[:] = np.array([0.2, -0.1, 0.05])[:, None, None]
    w0 = st.omega.copy()
    O.step(p, st, 2)
    assert np.abs(st.omega - w0).max() < 1e-15
    assert np.abs(st.force).max() < 1e-20
    assert np.abs(st.vel).max() < 1e-20


def test_decoupled_flow_stays_at_rest(oracle_lib):
    # inv_beta_v = 0 and f0 = 0: no force reaches the fluid, so the LB stays
    # exactly at rest and the EPD part runs alone (the no-LB case of Sec. 3).
    p = O.Params(nx=16, ny=8, ns=6, f0=0.0, inv_beta_v=0.0, noise_amp=1e-2)
    st = O.initial_state(p)
    O.step(p, st, 3)
    assert np.all(st.vel == 0)
    assert np.all(st.force == 0)


def test_hydrodynamics_changes_little(oracle_lib):
    # T13 (qualitative, Sec. 3): coupling to LB perturbs Phi_P only slightly.
    p = O.Params(nx=16, ny=16, ns=8, f0=0.0, noise_amp=1e-2)
    a = O.initial_state(p)
    b = O.initial_state(O.Params(**{**p.__dict__, "inv_beta_v": 0.0}))
    pb = O.Params(**{**p.__dict__, "inv_beta_v": 0.0})
    O.step(p, a, 5)
    O.step(pb, b, 5)
    d = np.abs((a.phi[0] + a.phi[1]) - (b.phi[0] + b.phi[1])).mean()
    s = O.sigma(p, a.phi)
    assert 0 < d < 1e-3 * s
