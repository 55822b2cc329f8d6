"""GPU D3Q19 collide-stream (the three-dimensional LB scheme named for the
extension to 3D) against the FP64 oracle: random states with ghost content
and forces for several relaxation sets and boxes, and 20 steps under the
reverse-Poiseuille force."""
import numpy as np
import pytest

import oracle as O
import paper_1804_02883_gb300 as P
from helpers import oracle_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build(oracle_lib):
    P.lib()


def _state(nz, ny, nx, seed):
    rng = np.random.default_rng(seed)
    C, W = O.D3Q19_C, O.D3Q19_W
    rho = 1 + 0.05 * rng.standard_normal((nz, ny, nx))
    u = 0.03 * rng.standard_normal((3, nz, ny, nx))
    cu = np.einsum("ia,a...->i...", C, u)
    uu = (u * u).sum(axis=0)
    eq = W[:, None, None, None] * rho * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * uu)
    pop = eq * (1 + 0.02 * rng.standard_normal((19, nz, ny, nx)))
    f = 1e-3 * rng.standard_normal((3, nz, ny, nx))
    return pop, f


@pytest.mark.parametrize("gam", [(0.0, 0.0, 0.0), (0.5, -0.25, 0.3), (-0.7, 0.2, -0.4)])
@pytest.mark.parametrize("nx,ny,nz", [(8, 8, 8), (16, 8, 4), (10, 12, 6)])
def test_d3q19_step_matches_oracle(gam, nx, ny, nz):
    r = P.RunParams(nx=nx, ny=ny, ns=8, precision=P.PLAIN_FP64, gamma_s=gam[0], gamma_b=gam[1], gamma_g=gam[2])
    pop, f = _state(nz, ny, nx, nx + ny + nz)
    got, gvel = P.lb3d_step(r, pop, f)
    want, wvel = O.lb3d_step(oracle_params(r), nz, pop, f)
    assert np.abs(got - want).max() < 1e-15
    assert np.abs(gvel - wvel).max() < 1e-15


def test_d3q19_twenty_steps_under_the_channel_force():
    r = P.RunParams(nx=8, ny=16, ns=8, precision=P.PLAIN_FP64, gamma_s=0.3, gamma_b=0.3, gamma_g=0.0, f0=1.0)
    p = oracle_params(r)
    nz = 4
    pop, _ = _state(nz, 16, 8, 5)
    f = np.zeros((3, nz, 16, 8))
    f[0] = np.array([O.poiseuille_force(p, y) for y in range(16)])[None, :, None]
    g, o = pop.copy(), pop.copy()
    for _ in range(20):
        g, gv = P.lb3d_step(r, g, f)
        o, ov = O.lb3d_step(p, nz, o, f)
    assert np.abs(g - o).max() < 1e-14
    assert np.abs(gv - ov).max() < 1e-14
    assert abs(g.sum() - pop.sum()) < 1e-11


def test_d3q19_rejects_bad_boxes():
    r = P.RunParams(nx=8, ny=8, ns=8, precision=P.PLAIN_FP64)
    with pytest.raises(P.EpdLbError):
        P.lb3d_step(r, np.zeros((19, 7, 8, 8)), np.zeros((3, 7, 8, 8)))
