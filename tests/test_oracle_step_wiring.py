"""Pins of the oracle's coupled step (App. C; Sec. 2, Eqs. (5), (19)-(20);
Eqs. (12), (14)) on how its parts are wired together.

The parts are pinned elsewhere (propagator T1-T5, mu, spectral operators,
force, LB closed forms).  Here one oracle step, taken from a flowing state,
is checked against relations that the paper fixes between the step's
inputs and outputs, each evaluated with numpy's FFT (not the oracle's):

1. Phi~ is the density of the auxiliary-convected field
   omega~ = omega - dt v . grad omega (App. C, item 1), not of omega;
2. omega(t+dt) - omega~ = -dt D_I Lap mu_I with mu at (Phi~, omega~)
   (Eq. (5); App. C, last item);
3. Phi(t+dt) is the density of omega(t+dt);
4. div f = -(1/(beta v)) sum_I (Phi_I(t+dt) - Phi~_I) / (D_I dt) and
   curl f = 0 (Eqs. (19)-(20), App. A), in units of f*;
5. the collision adds exactly f + f_P(y) to the momentum of every site and
   the velocity handed on is (j + (f + f_P)/2) / rho (Eq. (14), reading of
   the Dunweg-Ladd forcing).

Each check also runs on steps composed from the oracle's pinned parts with
one plausible wiring mistake, and must reject every one of them: the pair
of the force taken as Phi(t+dt) - Phi(t), mu evaluated at Phi(t), the
polymer force handed to LB with the wrong sign, solve #1 at omega instead
of omega~.
"""
import numpy as np
import pytest

import oracle as O
from paper_1804_02883_gb300 import workloads as W

CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])


def wavenumbers(p):
    """Continuum wavenumbers (ky[:, None], kx[None, :]) and masks of the
    Nyquist bins (reading: a first derivative drops them)."""
    kx = 2 * np.pi * np.fft.fftfreq(p.nx, d=p.dx)
    ky = 2 * np.pi * np.fft.fftfreq(p.ny, d=p.dx)
    nyq_x = np.zeros(p.nx, bool)
    nyq_y = np.zeros(p.ny, bool)
    if p.nx % 2 == 0:
        nyq_x[p.nx // 2] = True
    if p.ny % 2 == 0:
        nyq_y[p.ny // 2] = True
    return ky[:, None], kx[None, :], nyq_y[:, None], nyq_x[None, :]


def grad(p, f):
    ky, kx, ny_, nx_ = wavenumbers(p)
    fh = np.fft.fft2(f)
    gx = np.fft.ifft2(np.where(nx_, 0, 1j * kx) * fh).real
    gy = np.fft.ifft2(np.where(ny_, 0, 1j * ky) * fh).real
    return gx, gy


def lap(p, f):
    ky, kx, _, _ = wavenumbers(p)
    return np.fft.ifft2(-(kx ** 2 + ky ** 2) * np.fft.fft2(f)).real


def diffusivities(p):
    return np.array([p.d_p, p.d_p, p.d_s])


def omega_tilde_np(p, omega, vel):
    """App. C, item 1: omega~ = omega - dt v . grad omega, v = u_lat dx/dt."""
    v = vel * (p.dx / p.dt)
    out = np.empty_like(omega)
    for s in range(3):
        gx, gy = grad(p, omega[s])
        out[s] = omega[s] - p.dt * (v[0] * gx + v[1] * gy)
    return out


def flowing_state(seed=3):
    """A 16 x 32 state with a sheared flow, a non-uniform polymer force and
    populations off equilibrium (so that every part of the step matters)."""
    r = W.with_(W.plain_small(), nx=32, ny=16, ns=8, f0=40.0, noise_amp=0.0, phi_p=0.2)
    p = O.Params(**{k: getattr(r, k) for k in O.Params.__dataclass_fields__})
    omega = W.random_omega(p.ny, p.nx, seed=seed, amp=0.1)
    pop = W.random_populations(p.ny, p.nx, seed=seed + 1, amp=2e-3)
    vel = W.random_velocity(p.ny, p.nx, seed=seed + 2, amp=0.03)
    phi, q = O.solve(p, omega)
    return p, O.State(omega, pop, vel, phi, q, np.zeros((2, p.ny, p.nx)))


def copy_state(st):
    return O.State(*(np.array(a, copy=True) for a in (st.omega, st.pop, st.vel, st.phi, st.q, st.force)))


def oracle_step(p, st):
    """One step of the C oracle: (state before, state after, Phi~)."""
    before = copy_state(st)
    after = copy_state(st)
    pt = O.step(p, after, 1, phi_tilde_out=True)
    return before, after, pt


def composed_step(p, st, mistake):
    """One step composed from the oracle's pinned parts in the order of
    App. C, with one wiring mistake planted."""
    before = copy_state(st)
    wt = O.aux_convection(p, st.omega, st.vel)
    pt, _ = O.solve(p, st.omega if mistake == "solve1_at_omega" else wt)
    mu = O.mu(p, st.phi if mistake == "mu_at_phi_t" else pt, wt)
    om = O.diffusion_update(p, wt, mu)
    phi, q = O.solve(p, om)
    f = O.force(p, phi - (st.phi if mistake == "pair_phi_t" else pt))
    fl = -f if mistake == "force_sign" else f
    fp = np.array([O.poiseuille_force(p, y) for y in range(p.ny)])
    ftot = np.stack((fl[0] + fp[:, None], fl[1]))
    pop, vel = O.lb_step(p, st.pop, ftot)
    return before, O.State(om, pop, vel, phi, q, f), pt


MISTAKES = ["pair_phi_t", "mu_at_phi_t", "force_sign", "solve1_at_omega"]


# --- the five relations; each returns an error relative to its scale -------

def err_phi_tilde(p, before, after, pt):
    want, _ = O.solve(p, omega_tilde_np(p, before.omega, before.vel))
    return np.abs(pt - want).max() / np.abs(want - want.mean(axis=(1, 2), keepdims=True)).max()


def err_diffusion(p, before, after, pt):
    wt = omega_tilde_np(p, before.omega, before.vel)
    mu = O.mu(p, pt, wt)
    d = diffusivities(p)
    want = np.stack([wt[s] - p.dt * d[s] * lap(p, mu[s]) for s in range(3)])
    return np.abs(after.omega - want).max() / np.abs(after.omega - wt).max()


def err_solve2(p, before, after, pt):
    want, q = O.solve(p, after.omega)
    return max(np.abs(after.phi - want).max() / np.abs(want).max(), np.abs(after.q - q).max() / np.abs(q).max())


def err_force(p, before, after, pt):
    ky, kx, ny_, nx_ = wavenumbers(p)
    f = after.force / O.fstar_lattice(p)  # units of f*
    fx, fy = np.fft.fft2(f[0]), np.fft.fft2(f[1])
    div = 1j * kx * fx + 1j * ky * fy
    curl = 1j * kx * fy - 1j * ky * fx
    s = sum((after.phi[i] - pt[i]) / diffusivities(p)[i] for i in range(3))
    want = -p.inv_beta_v * np.fft.fft2(s) / p.dt
    keep = ~(ny_ | nx_)  # modes where neither first derivative is dropped
    keep[0, 0] = False
    scale = np.abs(want[keep]).max()
    return max(np.abs(div - want)[keep].max(), np.abs(curl)[keep].max()) / scale


def err_lb(p, before, after, pt):
    """Undo the streaming (post-collision n*_i(x) = n_i(x + c_i) after the
    step), then compare the momentum gained at every site with f + f_P and the
    velocity handed on with (j + f_tot / 2) / rho."""
    post = np.stack([np.roll(after.pop[i], (-CY[i], -CX[i]), axis=(0, 1)) for i in range(9)])
    rho = before.pop.sum(0)
    j0 = np.stack(((CX[:, None, None] * before.pop).sum(0), (CY[:, None, None] * before.pop).sum(0)))
    j1 = np.stack(((CX[:, None, None] * post).sum(0), (CY[:, None, None] * post).sum(0)))
    fp = np.array([O.poiseuille_force(p, y) for y in range(p.ny)])
    ftot = np.stack((after.force[0] + fp[:, None], after.force[1]))
    e_mom = np.abs(j1 - j0 - ftot).max() / np.abs(ftot).max()
    e_mass = np.abs(post.sum(0) - rho).max() / rho.max()
    u = (j0 + ftot / 2) / rho
    e_vel = np.abs(after.vel - u).max() / np.abs(u).max()
    return max(e_mom, e_mass * 1e4, e_vel)


CHECKS = {"phi_tilde": err_phi_tilde, "diffusion": err_diffusion, "solve2": err_solve2, "force": err_force,
          "lb": err_lb}
# which check each planted mistake must trip (others may trip too)
CAUGHT_BY = {"pair_phi_t": "force", "mu_at_phi_t": "diffusion", "force_sign": "lb", "solve1_at_omega": "phi_tilde"}


@pytest.mark.parametrize("name", sorted(CHECKS))
def test_oracle_step_satisfies_wiring(oracle_lib, name):
    p, st = flowing_state()
    before, after, pt = oracle_step(p, st)
    assert CHECKS[name](p, before, after, pt) < 1e-10, name


def test_composition_of_parts_is_the_oracle_step(oracle_lib):
    # the planted-mistake steps differ from the oracle's only where planted
    p, st = flowing_state()
    _, a, pa = oracle_step(p, st)
    _, b, pb = composed_step(p, st, None)
    for x, y in ((a.omega, b.omega), (a.phi, b.phi), (a.pop, b.pop), (a.vel, b.vel), (a.force, b.force), (pa, pb)):
        assert np.abs(x - y).max() <= 1e-15 * max(1.0, np.abs(y).max())


@pytest.mark.parametrize("mistake", MISTAKES)
def test_each_wiring_mistake_is_caught(oracle_lib, mistake):
    p, st = flowing_state()
    before, after, pt = composed_step(p, st, mistake)
    errs = {k: f(p, before, after, pt) for k, f in CHECKS.items()}
    assert errs[CAUGHT_BY[mistake]] > 1e-3, (mistake, errs)


def test_wiring_over_several_steps(oracle_lib):
    # the relations hold at every step of a short trajectory, not only the first
    p, st = flowing_state(seed=11)
    for _ in range(3):
        before, after, pt = oracle_step(p, st)
        for name, f in CHECKS.items():
            assert f(p, before, after, pt) < 1e-10, name
        st = after
