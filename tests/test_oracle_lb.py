"""Pins of the oracle's D2Q9 LB (Sec. 2, Eqs. (12), (14)-(16); Sec. 4,
Eqs. (23)-(24)): conservation (T9), the exact discrete reverse-Poiseuille
steady state (T10), identity with BGK + Guo forcing when all non-conserved
modes relax alike (T11), rest and uniform-flow invariance (T12), and the
shear viscosity of Eq. (16) from the decay of a shear wave."""
import numpy as np
import pytest

import oracle as O

CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
CS2 = 1 / 3


def equilibrium(rho, ux, uy):
    cu = CX[:, None, None] * ux[None] + CY[:, None, None] * uy[None]
    uu = ux ** 2 + uy ** 2
    return W[:, None, None] * rho[None] * (1 + cu / CS2 + cu ** 2 / (2 * CS2 ** 2) - uu[None] / (2 * CS2))


def stream(post):
    out = np.empty_like(post)
    for i in range(9):
        out[i] = np.roll(np.roll(post[i], CX[i], axis=1), CY[i], axis=0)
    return out


def random_state(p, rng, amp=0.05):
    rho = 1 + amp * rng.standard_normal((p.ny, p.nx))
    ux = amp * rng.standard_normal((p.ny, p.nx))
    uy = amp * rng.standard_normal((p.ny, p.nx))
    return equilibrium(rho, ux, uy) * (1 + 0.1 * rng.standard_normal((9, p.ny, p.nx)))


def test_conservation(oracle_lib):
    # T9: mass is conserved and total momentum changes by the total force.
    p = O.Params(nx=16, ny=8, gamma_s=-0.3, gamma_b=0.2, gamma_g=0.4)
    rng = np.random.default_rng(1)
    pop = random_state(p, rng)
    f = 1e-3 * rng.standard_normal((2, p.ny, p.nx))
    new, _ = O.lb_step(p, pop, f)
    assert abs(new.sum() - pop.sum()) < 1e-12
    for c, a in ((CX, 0), (CY, 1)):
        before = (c[:, None, None] * pop).sum()
        after = (c[:, None, None] * new).sum()
        assert abs(after - before - f[a].sum()) < 1e-12


@pytest.mark.parametrize("gamma", [0.0, 0.5, -0.5, 0.8])
def test_bgk_guo_identity(oracle_lib, gamma):
    # T11: relaxing every non-conserved mode by gamma is BGK with
    # tau = 1/(1-gamma) and Guo forcing (1 - 1/(2 tau)) F_i,
    #   F_i = w_i [(c_i - u).f / c_s^2 + (c_i.u)(c_i.f) / c_s^4],
    # written here population by population.
    p = O.Params(nx=8, ny=16, gamma_s=gamma, gamma_b=gamma, gamma_g=gamma)
    rng = np.random.default_rng(2)
    pop = random_state(p, rng)
    f = 1e-3 * rng.standard_normal((2, p.ny, p.nx))
    rho = pop.sum(0)
    ux = ((CX[:, None, None] * pop).sum(0) + f[0] / 2) / rho
    uy = ((CY[:, None, None] * pop).sum(0) + f[1] / 2) / rho
    tau = 1 / (1 - gamma)
    cu = CX[:, None, None] * ux + CY[:, None, None] * uy
    cf = CX[:, None, None] * f[0] + CY[:, None, None] * f[1]
    uf = ux * f[0] + uy * f[1]
    F = W[:, None, None] * ((cf - uf[None]) / CS2 + cu * cf / CS2 ** 2)
    post = pop - (pop - equilibrium(rho, ux, uy)) / tau + (1 - 1 / (2 * tau)) * F
    want = stream(post)
    got, vel = O.lb_step(p, pop, f)
    assert np.abs(got - want).max() < 1e-15 * 8
    assert np.abs(vel[0] - ux).max() < 1e-16 * 8


@pytest.mark.parametrize("u0", [(0.0, 0.0), (0.05, -0.03)])
def test_rest_and_uniform_flow_invariant(oracle_lib, u0):
    # T12: a uniform equilibrium without force is a fixed point.
    p = O.Params(nx=8, ny=8, gamma_s=0.3, gamma_b=-0.2, gamma_g=0.1)
    rho = np.full((p.ny, p.nx), 1.02)
    pop = equilibrium(rho, np.full_like(rho, u0[0]), np.full_like(rho, u0[1]))
    cur = pop.copy()
    for _ in range(10):
        cur, vel = O.lb_step(p, cur, np.zeros((2, p.ny, p.nx)))
    assert np.abs(cur - pop).max() < 1e-15 * 10
    assert np.abs(vel[0] - u0[0]).max() < 1e-14


@pytest.mark.parametrize("gamma", [0.0, 0.5, -0.5])
def test_reverse_poiseuille_discrete_steady_state(oracle_lib, gamma):
    # T10: with the body force of Eq. (23) the LB relaxes to
    #   u(y) = v(y + 1/2) + f_P(y) (1 - 1/(8 eta)),
    # v the flow field of Eq. (24) and eta from Eq. (16) -- the exact steady
    # state of the scheme for gamma_g = 0 (derivation in the design notes).
    p = O.Params(nx=4, ny=16, gamma_s=gamma, gamma_b=gamma, gamma_g=0.0)
    p.f0 = 1e-6 / O.fstar_lattice(p)
    omega, pop, vel = O.init(p)
    fP = np.array([O.poiseuille_force(p, y) for y in range(p.ny)])
    ftot = np.zeros((2, p.ny, p.nx))
    ftot[0] = fP[:, None]
    for _ in range(4000):
        pop, vel = O.lb_step(p, pop, ftot)
    want = np.array([O.discrete_profile(p, y) for y in range(p.ny)])
    assert np.abs(vel[0] - want[:, None]).max() < 1e-9 * np.abs(want).max()
    assert np.abs(vel[1]).max() < 1e-14
    assert abs(pop.sum() - p.n) < 1e-10  # round-off over 4000 steps


def test_reverse_poiseuille_continuum_limit(oracle_lib):
    # The discrete profile approaches Eq. (24) with a relative deviation
    # O(1/L_y^2).
    devs = []
    for ny in (16, 32, 64, 128):
        p = O.Params(nx=4, ny=ny, f0=1.0)
        v = np.array([O.discrete_profile(p, y) for y in range(ny)])
        c = np.array([O.flow_profile(p, y + 0.5) for y in range(ny)])
        devs.append(np.abs(v - c).max() / np.abs(c).max())
    for a, b in zip(devs[:-1], devs[1:]):
        assert 3.5 < a / b < 4.5
    # Eq. (24) vanishes at y = 0, L_y/2 and L_y and peaks at f0 L_y^2/(32 eta)
    p = O.Params(nx=4, ny=64, f0=1.0)
    a = p.f0 * O.fstar_lattice(p)
    assert abs(O.flow_profile(p, 0.0)) < 1e-20 and abs(O.flow_profile(p, 32.0)) < 1e-20
    assert abs(O.flow_profile(p, 48.0) - a * 64 ** 2 / (32 * O.eta(p))) < 1e-15


@pytest.mark.parametrize("gamma", [0.0, 0.5, -0.5])
def test_shear_viscosity_from_shear_wave(oracle_lib, gamma):
    # A transverse wave u_x = U sin(k y) decays as exp(-nu k^2 t) with
    # nu = eta/rho and eta = (rho c_s^2 / 2)(1 + gamma_s)/(1 - gamma_s), Eq. (16).
    p = O.Params(nx=4, ny=128, gamma_s=gamma, gamma_b=gamma)
    k = 2 * np.pi / p.ny
    y = np.arange(p.ny)
    rho = np.ones((p.ny, p.nx))
    ux = 1e-4 * np.sin(k * y)[:, None] * np.ones((1, p.nx))
    pop = equilibrium(rho, ux, np.zeros_like(ux))
    zero = np.zeros((2, p.ny, p.nx))

    def amp(v):
        return 2 * (v[0, :, 0] * np.sin(k * y)).mean()

    for _ in range(50):
        pop, vel = O.lb_step(p, pop, zero)
    a1 = amp(vel)
    for _ in range(400):
        pop, vel = O.lb_step(p, pop, zero)
    a2 = amp(vel)
    nu = -np.log(a2 / a1) / 400 / k ** 2
    assert abs(nu / O.eta(p) - 1) < 2e-3
