"""The segment-symmetric junction rule (junction_rule = 1: both half-steps
of a contour interval use its block's field, Sec. 2 and Eq. (8)) on every
solve path of the GPU against the FP64 oracle: radix-2 streaming (FP64),
cluster-resident (MIXED), radix-8 streaming (MIXED), mixed-radix (the paper's
150 x 150 grid, N_s = 17, q_A = 0.882), the differential second solve of a
coupled step, and the 3D solve."""
import numpy as np
import pytest

import oracle as O
import paper_1804_02883_gb300 as P
from paper_1804_02883_gb300 import workloads as W
from helpers import fluct_err, oracle_params, rel_err

pytestmark = pytest.mark.gpu

TOL = {P.PLAIN_FP64: 1e-10, P.MIXED_FP32: 2e-5}


@pytest.fixture(scope="module", autouse=True)
def _build(oracle_lib):
    P.lib()


@pytest.mark.parametrize("prec,ny,nx,ns,f_a", [
    (P.PLAIN_FP64, 32, 64, 12, 0.25),      # radix-2 streaming
    (P.PLAIN_FP64, 150, 150, 17, 0.882),   # mixed-radix, the paper's system
    (P.MIXED_FP32, 64, 64, 16, 0.25),      # cluster-resident
    (P.MIXED_FP32, 256, 512, 64, 0.3),     # cluster-resident, the benchmark grid
    (P.MIXED_FP32, 64, 1024, 8, 0.375),    # radix-8 streaming
    (P.MIXED_FP32, 96, 60, 10, 0.3),       # mixed-radix in FP32
])
def test_segment_symmetric_solve_matches_oracle(prec, ny, nx, ns, f_a):
    r = P.RunParams(nx=nx, ny=ny, ns=ns, precision=prec, f_a=f_a, phi_p=0.2, junction_rule=1)
    h = P.EpdLb([r])
    om = W.random_omega(ny, nx, seed=ny + nx + ns, amp=0.2)
    phi, q = h.solve(0, om)
    ophi, oq = O.solve(oracle_params(r), om)
    assert rel_err(q, oq) < TOL[prec]
    for s in range(3):
        assert rel_err(phi[s], ophi[s]) < TOL[prec], s
    # the rule matters on this field: the literal reading differs
    lit, _ = O.solve(oracle_params(W.with_(r, junction_rule=0)), om)
    assert rel_err(lit, ophi) > 10 * TOL[prec]
    h.close()


@pytest.mark.parametrize("ny,nx,ns", [(64, 64, 16), (64, 128, 10)])
def test_segment_symmetric_coupled_step_differential_solve(ny, nx, ns):
    # one coupled step from a random state on cluster grids: the second solve
    # is the differential one, with the junction node's mixed factor E_A E_B
    r = P.RunParams(nx=nx, ny=ny, ns=ns, precision=P.MIXED_FP32, f_a=0.3, phi_p=0.2, f0=2.0, junction_rule=1)
    omega = W.random_omega(ny, nx, seed=31, amp=0.05)
    pop = W.random_populations(ny, nx, seed=32)
    vel = W.random_velocity(ny, nx, seed=33, amp=0.02)
    h = P.EpdLb([r])
    assert h.tiles(0)["path"] == 2 and h.tiles(0)["differential"]
    h.set_state(0, omega, pop, vel)
    h.step(1)
    p = oracle_params(r)
    phi0, q0 = O.solve(p, omega)
    st = O.State(omega.copy(), pop.copy(), vel.copy(), phi0, q0, np.zeros((2, ny, nx)))
    O.step(p, st)
    gom, gpop, gvel = h.get_state(0)
    gphi, gq = h.densities(0)
    assert rel_err(gphi, st.phi) < 2e-6
    assert rel_err(gq, st.q) < 2e-6
    assert fluct_err(gom, st.omega) < 2e-6
    assert rel_err(gvel, st.vel) < 1e-5
    h.close()


def test_segment_symmetric_fp64_steps_match_oracle():
    r = W.with_(W.plain_small(), nx=32, ny=32, ns=12, f_a=0.25, f0=20.0, noise_amp=1e-2, junction_rule=1)
    h = P.EpdLb([r])
    p = oracle_params(r)
    st = O.initial_state(p)
    h.step(5)
    O.step(p, st, 5)
    gphi, _ = h.densities(0)
    assert rel_err(gphi, st.phi) < 1e-10
    assert fluct_err(h.get_state(0)[0], st.omega) < 1e-9
    h.close()


@pytest.mark.parametrize("prec", [P.PLAIN_FP64, P.MIXED_FP32])
def test_segment_symmetric_solve3d(prec):
    r = P.RunParams(nx=16, ny=8, ns=8, precision=prec, f_a=0.375, phi_p=0.2, junction_rule=1)
    nz = 16
    rng = np.random.default_rng(4)
    om = 0.2 * rng.standard_normal((3, nz, 8, 16))
    phi, q = P.prop_solve3d(r, om)
    ophi, oq = O.solve3d(oracle_params(r), nz, om)
    tol = 1e-12 if prec == P.PLAIN_FP64 else 2e-5
    assert rel_err(q, oq) < tol
    assert rel_err(phi, ophi) < tol


def test_junction_rule_is_validated():
    with pytest.raises(P.EpdLbError) as ei:
        P.EpdLb([P.RunParams(nx=32, ny=32, ns=8, junction_rule=2)])
    assert ei.value.code == -1
