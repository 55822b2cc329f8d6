"""Pins of the oracle's D3Q19 collide-stream (the three-dimensional scheme
named in Sec. 2 for the extension to 3D): conservation, the BGK + Guo
identity at gamma = 0, stationary equilibria, and the exact discrete
reverse-Poiseuille steady state of the D2Q9 scheme, which a flow uniform in
z must keep."""
import numpy as np
import pytest

import oracle as O

C, W = O.D3Q19_C, O.D3Q19_W
CS2 = 1.0 / 3.0


def _eq(rho, u):
    cu = np.einsum("ia,a...->i...", C, u)
    uu = (u * u).sum(axis=0)
    return W[:, None, None, None] * rho * (1 + cu / CS2 + cu * cu / (2 * CS2 ** 2) - uu / (2 * CS2))


def _random_state(p, nz, seed):
    rng = np.random.default_rng(seed)
    rho = 1 + 0.05 * rng.standard_normal((nz, p.ny, p.nx))
    u = 0.03 * rng.standard_normal((3, nz, p.ny, p.nx))
    pop = _eq(rho, u) * (1 + 0.02 * rng.standard_normal((19, nz, p.ny, p.nx)))  # with ghost content
    f = 1e-3 * rng.standard_normal((3, nz, p.ny, p.nx))
    return pop, f


@pytest.mark.parametrize("g", [0.0, 0.5, -0.7])
def test_d3q19_conserves_mass_and_adds_the_force(oracle_lib, g):
    p = O.Params(nx=6, ny=4, gamma_s=g, gamma_b=-g / 2, gamma_g=g / 3)
    nz = 5
    pop, f = _random_state(p, nz, 1)
    new, vel = O.lb3d_step(p, nz, pop, f)
    assert abs(new.sum() - pop.sum()) < 1e-12
    j0 = np.einsum("ia,i...->a...", C, pop).reshape(3, -1).sum(axis=1)
    j1 = np.einsum("ia,i...->a...", C, new).reshape(3, -1).sum(axis=1)
    assert np.abs(j1 - j0 - f.sum(axis=(1, 2, 3))).max() < 1e-12
    # u = (j + f/2) / rho at the collision
    rho = pop.sum(axis=0)
    u = (np.einsum("ia,i...->a...", C, pop) + 0.5 * f) / rho
    assert np.abs(vel - u).max() < 1e-15


def test_d3q19_gamma_zero_is_bgk_tau_one_with_guo_forcing(oracle_lib):
    # gamma = 0: n* = n_eq(rho, u) + (1 - 1/2) F_i, Guo's forcing term
    # F_i = w_i [(c_i - u)/c_s^2 + (c_i . u) c_i / c_s^4] . f, then streaming
    p = O.Params(nx=6, ny=4, gamma_s=0.0, gamma_b=0.0, gamma_g=0.0)
    nz = 4
    pop, f = _random_state(p, nz, 2)
    new, _ = O.lb3d_step(p, nz, pop, f)
    rho = pop.sum(axis=0)
    u = (np.einsum("ia,i...->a...", C, pop) + 0.5 * f) / rho
    cu = np.einsum("ia,a...->i...", C, u)
    cf = np.einsum("ia,a...->i...", C, f)
    uf = (u * f).sum(axis=0)
    F = W[:, None, None, None] * ((cf - uf) / CS2 + cu * cf / CS2 ** 2)
    post = _eq(rho, u) + 0.5 * F
    want = np.empty_like(post)
    for i, c in enumerate(C):
        want[i] = np.roll(post[i], shift=(c[2], c[1], c[0]), axis=(0, 1, 2))
    assert np.abs(new - want).max() < 1e-14


@pytest.mark.parametrize("g", [0.0, 0.6])
def test_d3q19_equilibria_are_stationary(oracle_lib, g):
    p = O.Params(nx=4, ny=6, gamma_s=g, gamma_b=g, gamma_g=g)
    nz = 3
    u = np.zeros((3, nz, p.ny, p.nx))
    u[0], u[1], u[2] = 0.04, -0.02, 0.01
    pop = _eq(np.ones((nz, p.ny, p.nx)), u)
    new, _ = O.lb3d_step(p, nz, pop, np.zeros((3, nz, p.ny, p.nx)))
    assert np.abs(new - pop).max() < 1e-15


@pytest.mark.parametrize("g", [0.0, 0.5, -0.5])
def test_d3q19_relaxes_to_the_exact_discrete_poiseuille_state(oracle_lib, g):
    # the D2Q9 steady state u(y) = v(y + 1/2) + f_P(y) (1 - 1/(8 eta)) under the
    # reverse-Poiseuille force of Eq. (23) is the steady state of the scheme's
    # moment balance; a flow uniform in x and z on D3Q19 reaches it as well
    p = O.Params(nx=4, ny=16, gamma_s=g, gamma_b=g, gamma_g=0.0)
    p.f0 = 1e-6 / O.fstar_lattice(p)
    nz = 3
    fy = np.array([O.poiseuille_force(p, y) for y in range(p.ny)])
    v = np.array([O.discrete_profile(p, y) for y in range(p.ny)])
    u = np.zeros((3, nz, p.ny, p.nx))
    u[0] = (v - 0.5 * fy)[None, :, None]
    pop = _eq(np.ones((nz, p.ny, p.nx)), u)
    f = np.zeros((3, nz, p.ny, p.nx))
    f[0] = fy[None, :, None]
    for _ in range(3000):
        pop, vel = O.lb3d_step(p, nz, pop, f)
    assert np.abs(vel[0] - v[None, :, None]).max() < 1e-9 * np.abs(v).max()
    assert np.abs(vel[1:]).max() < 1e-14
