"""GPU single-chain solve on 3D boxes (Eqs. (6)-(11) with
|k|^2 = kx^2 + ky^2 + kz^2, the extension named in Sec. 2 and Sec. 5)
against the FP64 oracle: power-of-two and mixed-radix axes, both
precisions, the homogeneous closed form and exact masses."""
import numpy as np
import pytest

import oracle as O
import paper_1804_02883_gb300 as P
from helpers import oracle_params, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build(oracle_lib):
    P.lib()


@pytest.mark.parametrize("prec", [P.PLAIN_FP64, P.MIXED_FP32])
@pytest.mark.parametrize("nx,ny,nz,ns", [(16, 8, 32, 8), (32, 32, 32, 12), (10, 12, 30, 7), (64, 32, 16, 16),
                                          (8, 8, 2, 6)])
def test_solve3d_matches_oracle(prec, nx, ny, nz, ns):
    r = P.RunParams(nx=nx, ny=ny, ns=ns, precision=prec, f_a=0.4, phi_p=0.2)
    rng = np.random.default_rng(nx * ny + nz)
    om = 0.1 * rng.standard_normal((3, nz, ny, nx))
    phi, q = P.prop_solve3d(r, om)
    ophi, oq = O.solve3d(oracle_params(r), nz, om)
    tol = 1e-12 if prec == P.PLAIN_FP64 else 2e-5
    assert rel_err(q, oq) < tol
    for s in range(3):
        assert rel_err(phi[s], ophi[s]) < tol, s


@pytest.mark.parametrize("prec", [P.PLAIN_FP64, P.MIXED_FP32])
def test_solve3d_homogeneous_and_masses(prec):
    r = P.RunParams(nx=32, ny=16, ns=10, precision=prec, f_a=0.3, phi_p=0.25)
    nz = 24
    phi, q = P.prop_solve3d(r, np.full((3, nz, 16, 32), 0.2))
    fa = round(0.3 * 10) / 10
    tol = 1e-14 if prec == P.PLAIN_FP64 else 1e-6
    assert np.abs(phi[0] - 0.25 * fa).max() < tol and np.abs(phi[2] - 0.75).max() < tol
    rng = np.random.default_rng(7)
    phi, _ = P.prop_solve3d(r, 0.3 * rng.standard_normal((3, nz, 16, 32)))
    assert abs(phi[0].mean() - 0.25 * fa) < (1e-13 if prec == P.PLAIN_FP64 else 1e-7)


def test_solve3d_rejects_unsupported_boxes():
    r = P.RunParams(nx=32, ny=32, ns=8, precision=P.PLAIN_FP64)
    for nz in (7, 14, 4096):
        with pytest.raises(P.EpdLbError):
            P.epd_prop_solve3d_workspace_bytes(r, nz)
    with pytest.raises(P.EpdLbError):  # more than 2^22 sites
        P.epd_prop_solve3d_workspace_bytes(P.RunParams(nx=256, ny=256, ns=8), 128)
    assert P.epd_prop_solve3d_workspace_bytes(P.RunParams(nx=128, ny=128, ns=8), 128) > 0
