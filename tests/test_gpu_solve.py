"""GPU single-chain solve (Sec. 2, Eqs. (6)-(11)) against the FP64 oracle and
against the closed forms the oracle is pinned to."""
import numpy as np
import pytest

import oracle as O
import paper_1804_02883_gb300 as P
from paper_1804_02883_gb300 import workloads as W
from helpers import oracle_params, rel_err

pytestmark = pytest.mark.gpu

TOL = {P.PLAIN_FP64: 1e-10, P.MIXED_FP32: 2e-5}


@pytest.fixture(scope="module", autouse=True)
def _build(oracle_lib):
    P.lib()


# includes every grid of the cluster-resident solve (MIXED_FP32), grids of
# the radix-8 streaming passes (MIXED_FP32, 64..2048 points per axis, no
# cluster shape) and grids of the radix-2 streaming passes
SHAPES = [(8, 8, 4), (16, 32, 8), (64, 64, 32), (32, 256, 16), (256, 16, 12), (8, 2048, 6), (1024, 8, 10),
          (64, 128, 10), (128, 64, 14), (128, 128, 16), (256, 128, 32), (128, 256, 12), (128, 512, 24),
          (512, 128, 8), (256, 256, 20), (256, 512, 64), (512, 256, 8),
          (64, 1024, 8), (1024, 64, 6), (512, 512, 8), (128, 2048, 4), (2048, 64, 4)]


@pytest.mark.parametrize("prec", [P.PLAIN_FP64, P.MIXED_FP32])
@pytest.mark.parametrize("ny,nx,ns", SHAPES)
def test_solve_matches_oracle(prec, ny, nx, ns):
    r = P.RunParams(nx=nx, ny=ny, ns=ns, precision=prec, f_a=0.4, phi_p=0.25)
    h = P.EpdLb([r])
    om = W.random_omega(ny, nx, seed=ny * 7 + nx + ns)
    phi, q = h.solve(0, om)
    ophi, oq = O.solve(oracle_params(r), om)
    assert rel_err(q, oq) < TOL[prec]
    for s in range(3):
        assert rel_err(phi[s], ophi[s]) < TOL[prec], s
    h.close()


@pytest.mark.parametrize("prec,nx,ny", [(P.PLAIN_FP64, 32, 16), (P.MIXED_FP32, 64, 64)])
@pytest.mark.parametrize("f_a,ns", [(0.0, 8), (1.0, 8), (0.3, 128), (0.882, 18), (0.5, 2)])
def test_solve_block_boundaries(prec, nx, ny, f_a, ns):
    # homopolymer limits and N_A at either end of the chain; the MIXED grid
    # takes the cluster-resident solve
    r = P.RunParams(nx=nx, ny=ny, ns=ns, precision=prec, f_a=f_a, phi_p=0.15)
    h = P.EpdLb([r])
    om = W.random_omega(ny, nx, seed=ns)
    phi, q = h.solve(0, om)
    ophi, oq = O.solve(oracle_params(r), om)
    assert rel_err(phi, ophi) < TOL[prec]
    assert abs(phi[0].mean() + phi[1].mean() - r.phi_p) < (1e-13 if prec == P.PLAIN_FP64 else 1e-7)
    h.close()


@pytest.mark.parametrize("prec", [P.PLAIN_FP64, P.MIXED_FP32])
def test_solve_at_the_largest_grid(prec):
    # 2048 x 2048, the largest grid the library takes (radix-2 FP64 and
    # radix-8 FP32 streaming passes), a short chain so that the oracle
    # finishes in seconds
    r = P.RunParams(nx=2048, ny=2048, ns=4, precision=prec, f_a=0.5, phi_p=0.2)
    h = P.EpdLb([r])
    om = W.random_omega(2048, 2048, seed=99, amp=0.05)
    phi, q = h.solve(0, om)
    ophi, oq = O.solve(oracle_params(r), om)
    assert rel_err(q, oq) < TOL[prec]
    assert rel_err(phi, ophi) < TOL[prec]
    h.close()


@pytest.mark.parametrize("prec", [P.PLAIN_FP64, P.MIXED_FP32])
def test_homogeneous_closed_form(prec):
    # T1 on the GPU: Phi_A = phi_p N_A/N_s, Phi_B = phi_p (N_s-N_A)/N_s, Phi_S = 1 - phi_p
    r = P.RunParams(nx=64, ny=32, ns=16, precision=prec, f_a=0.5, phi_p=0.2)
    h = P.EpdLb([r])
    om = np.empty((3, 32, 64))
    om[0], om[1], om[2] = 0.3, -0.2, 0.1
    phi, q = h.solve(0, om)
    tol = 1e-13 if prec == P.PLAIN_FP64 else 1e-6
    assert np.abs(phi[0] / 0.1 - 1).max() < tol
    assert np.abs(phi[1] / 0.1 - 1).max() < tol
    assert np.abs(phi[2] / 0.8 - 1).max() < tol
    ds = 1 / 16
    node = np.array([0.3 if j < 8 else -0.2 for j in range(17)])  # N_A = 8
    want_qp = np.exp(-17 * ds * (node[0] / 2 + node[1:16].sum() + node[16] / 2))
    assert abs(q[0] / want_qp - 1) < tol
    h.close()


@pytest.mark.parametrize("prec", [P.PLAIN_FP64, P.MIXED_FP32])
def test_mass_exact_for_random_fields(prec):
    # T5 on the GPU
    r = P.RunParams(nx=128, ny=64, ns=20, precision=prec, f_a=0.35, phi_p=0.15)
    h = P.EpdLb([r])
    om = W.random_omega(64, 128, seed=3, amp=0.3)
    phi, _ = h.solve(0, om)
    tol = 1e-13 if prec == P.PLAIN_FP64 else 1e-6
    assert abs((phi[0].mean() + phi[1].mean()) / r.phi_p - 1) < tol
    assert abs(phi[2].mean() / (1 - r.phi_p) - 1) < 1e-13
    h.close()


def test_debye_linear_response_on_gpu():
    # T3 on the GPU: cos(kx) coefficient of Phi_P - phi_p within 2e-4 of the
    # Debye prediction at N_s = 128 (the scheme's O(ds^2) error).
    eps = 1e-7
    r = P.RunParams(nx=32, ny=8, ns=128, precision=P.PLAIN_FP64, f_a=0.5, phi_p=0.3)
    h = P.EpdLb([r])
    x = np.arange(32) / 3.0
    k = 2 * np.pi * 2 / (32 / 3.0)
    w = np.broadcast_to(eps * np.cos(k * x)[None, :], (8, 32))
    om = np.stack([w, w, np.zeros_like(w)])
    phi, _ = h.solve(0, om)
    coef = 2 * ((phi[0] + phi[1] - 0.3) * np.cos(k * x)[None, :]).mean()
    xx = k * k
    want = -0.3 * 17 * eps * 2 * (np.exp(-xx) + xx - 1) / xx ** 2
    assert abs(coef / want - 1) < 2e-4
    h.close()


@pytest.mark.parametrize("prec", [P.PLAIN_FP64, P.MIXED_FP32])
def test_stateless_solve_entry_point(prec):
    import torch
    r = P.RunParams(nx=64, ny=32, ns=12, precision=prec, f_a=0.5, phi_p=0.2)
    om = W.random_omega(32, 64, seed=11)
    nb = P.epd_prop_solve_workspace_bytes(r)
    ws = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
    wptr = (ws.data_ptr() + 255) & ~255
    om_d = torch.from_numpy(om).cuda()
    phi_d = torch.empty_like(om_d)
    q_d = torch.empty(2, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    P.epd_prop_solve(r, om_d.data_ptr(), phi_d.data_ptr(), q_d.data_ptr(), wptr, nb, 0)
    torch.cuda.synchronize()
    ophi, oq = O.solve(oracle_params(r), om)
    assert rel_err(phi_d.cpu().numpy(), ophi) < TOL[prec]
    assert rel_err(q_d.cpu().numpy(), oq) < TOL[prec]
