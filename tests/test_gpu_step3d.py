"""GPU coupled step on 3D boxes against the FP64 oracle: random states with
flow and polymer force on power-of-two and mixed-radix boxes, several steps
under the reverse-Poiseuille force, both solve precisions."""
import numpy as np
import pytest

import oracle as O
import paper_1804_02883_gb300 as P
from helpers import fluct_err, oracle_params, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build(oracle_lib):
    P.lib()


def _state(nz, ny, nx, seed):
    rng = np.random.default_rng(seed)
    C, W = O.D3Q19_C, O.D3Q19_W
    om = 0.05 * rng.standard_normal((3, nz, ny, nx))
    u = 0.01 * rng.standard_normal((3, nz, ny, nx))
    cu = np.einsum("ia,a...->i...", C, u)
    pop = W[:, None, None, None] * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * (u * u).sum(axis=0))
    return om, pop, u


@pytest.mark.parametrize("nx,ny,nz,ns", [(16, 8, 8, 6), (8, 12, 10, 5), (32, 16, 8, 8)])
def test_step3d_matches_oracle(nx, ny, nz, ns):
    r = P.RunParams(nx=nx, ny=ny, ns=ns, precision=P.PLAIN_FP64, f_a=0.5, phi_p=0.2, f0=5.0)
    om, pop, vel = _state(nz, ny, nx, nx + ny + nz)
    g = P.step3d(r, om, pop, vel)
    o = O.step3d(oracle_params(r), nz, om, pop, vel)
    gom, gpop, gvel, gphi, gq, gf = g
    oom, opop, ovel, ophi, oq, of = o
    assert fluct_err(gom, oom) < 1e-10
    assert rel_err(gphi, ophi) < 1e-10
    assert rel_err(gq, oq) < 1e-12
    assert rel_err(gf, of) < 1e-9
    assert np.abs(gpop - opop).max() < 1e-14
    assert rel_err(gvel, ovel) < 1e-9


def test_three_steps_and_mixed_solves():
    nx, ny, nz = 16, 16, 8
    base = P.RunParams(nx=nx, ny=ny, ns=8, precision=P.PLAIN_FP64, f_a=0.5, phi_p=0.2, f0=5.0)
    om, pop, vel = _state(nz, ny, nx, 3)
    p = oracle_params(base)
    o = (om, pop, vel)
    for _ in range(3):
        o = O.step3d(p, nz, *o[:3])
    g = P.step3d(base, om, pop, vel, nsteps=3)
    assert fluct_err(g[0], o[0]) < 1e-10 and rel_err(g[3], o[3]) < 1e-10
    assert np.abs(g[1] - o[1]).max() < 1e-14
    # FP32 solves inside the same step
    m = P.step3d(P.RunParams(**{**base.__dict__, "precision": P.MIXED_FP32}), om, pop, vel, nsteps=3)
    assert fluct_err(m[0], o[0]) < 2e-5 and rel_err(m[3], o[3]) < 2e-5
