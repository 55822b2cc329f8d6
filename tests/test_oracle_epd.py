"""Pins of the oracle's EPD pieces: the chemical potential (derivative of the
free energy of Eq. (1)), spectral derivatives, the auxiliary convection of
omega (App. C), the diffusion step of Eq. (5), and the force reconstruction
of Eqs. (19)-(20) (T7: divergence, curl, closed form)."""
import numpy as np

import oracle as O


def test_mu_is_derivative_of_free_energy_density(oracle_lib):
    # The local part of Eq. (1):
    #   h = 1/2 sum_{I != J} chi_IJ Phi_I Phi_J - sum_I omega_I Phi_I
    #       + kappa_H/2 (sum_I Phi_I - 1)^2
    # differentiated numerically (central differences) at a random point.
    p = O.Params(nx=2, ny=2)
    chi = {(0, 1): p.chi_ab, (0, 2): p.chi_as, (1, 2): p.chi_bs}

    def h(ph, om):
        e = 0.0
        for I in range(3):
            for J in range(3):
                if I != J:
                    e += 0.5 * chi[tuple(sorted((I, J)))] * ph[I] * ph[J]
        return e - np.dot(om, ph) + 0.5 * p.kappa_h * (ph.sum() - 1) ** 2

    rng = np.random.default_rng(1)
    phi = rng.uniform(0.05, 0.8, size=(3, p.ny, p.nx))
    om = rng.normal(size=(3, p.ny, p.nx))
    mu = O.mu(p, phi, om)
    d = 1e-6
    for s in range(p.n):
        ph = phi.reshape(3, -1)[:, s].copy()
        o = om.reshape(3, -1)[:, s]
        for I in range(3):
            a, b = ph.copy(), ph.copy()
            a[I] += d
            b[I] -= d
            num = (h(a, o) - h(b, o)) / (2 * d)
            assert abs(num - mu.reshape(3, -1)[I, s]) < 1e-8


def _grid(p):
    x = np.arange(p.nx) * p.dx
    y = np.arange(p.ny) * p.dx
    return x[None, :], y[:, None]


def test_spectral_derivatives_of_modes(oracle_lib):
    p = O.Params(nx=16, ny=8)
    x, y = _grid(p)
    kx = 2 * np.pi * 3 / (p.nx * p.dx)
    ky = 2 * np.pi * 1 / (p.ny * p.dx)
    f = np.cos(kx * x + ky * y)
    assert np.abs(O.spectral_op(p, f, 0, 1) + kx * np.sin(kx * x + ky * y)).max() < 1e-12
    assert np.abs(O.spectral_op(p, f, 1, 1) + ky * np.sin(kx * x + ky * y)).max() < 1e-12
    assert np.abs(O.spectral_op(p, f, 0, 2) + kx ** 2 * f).max() < 1e-11
    assert np.abs(O.spectral_op(p, f, 2, 0) + (kx ** 2 + ky ** 2) * f).max() < 1e-11
    # Nyquist mode along x: zeroed in the first derivative, kept in the Laplacian
    kn = np.pi / p.dx
    fn = np.broadcast_to(np.cos(kn * x), (p.ny, p.nx))
    assert np.abs(O.spectral_op(p, fn, 0, 1)).max() < 1e-12
    assert np.abs(O.spectral_op(p, fn, 2, 0) + kn ** 2 * fn).max() < 1e-10


def test_aux_convection_closed_form(oracle_lib):
    p = O.Params(nx=16, ny=32)
    x, y = _grid(p)
    modes = [(1, 2), (3, 0), (0, 5)]
    omega = np.empty((3, p.ny, p.nx))
    grads = []
    for s, (mx, my) in enumerate(modes):
        kx = 2 * np.pi * mx / (p.nx * p.dx)
        ky = 2 * np.pi * my / (p.ny * p.dx)
        omega[s] = 0.01 * np.cos(kx * x + ky * y)
        grads.append((-0.01 * kx * np.sin(kx * x + ky * y), -0.01 * ky * np.sin(kx * x + ky * y)))
    rng = np.random.default_rng(2)
    vel = rng.uniform(-0.05, 0.05, size=(2, p.ny, p.nx))
    got = O.aux_convection(p, omega, vel)
    vs = p.dx / p.dt
    for s in range(3):
        want = omega[s] - p.dt * vs * (vel[0] * grads[s][0] + vel[1] * grads[s][1])
        assert np.abs(got[s] - want).max() < 1e-14


def test_diffusion_update_closed_form(oracle_lib):
    p = O.Params(nx=16, ny=16)
    x, y = _grid(p)
    kx = 2 * np.pi * 2 / (p.nx * p.dx)
    ky = 2 * np.pi * 3 / (p.ny * p.dx)
    mu = np.stack([np.cos(kx * x + 0 * y), np.sin(ky * y + 0 * x), np.cos(kx * x + ky * y)])
    wt = np.random.default_rng(3).normal(size=(3, p.ny, p.nx))
    got = O.diffusion_update(p, wt, mu)
    lam = [kx ** 2, ky ** 2, kx ** 2 + ky ** 2]
    dd = [p.d_p, p.d_p, p.d_s]
    for s in range(3):
        assert np.abs(got[s] - (wt[s] + p.dt * dd[s] * lam[s] * mu[s])).max() < 1e-12


def test_fstar_in_lattice_units(oracle_lib):
    # f* = rho R_G / tau^2 with dx = R_G/3, dt = 0.002 tau: 3 * 0.002^2
    assert abs(O.fstar_lattice(O.Params()) - 1.2e-5) < 1e-20


def test_force_single_mode_closed_form(oracle_lib):
    # T7: dPhi_A = a cos(k.r) gives f = -(1/beta v)/(D_A dt) a k sin(k.r)/|k|^2
    p = O.Params(nx=16, ny=8, inv_beta_v=0.7)
    x, y = _grid(p)
    kx = 2 * np.pi * 2 / (p.nx * p.dx)
    ky = 2 * np.pi * 1 / (p.ny * p.dx)
    a = 1e-4
    dphi = np.zeros((3, p.ny, p.nx))
    dphi[0] = a * np.cos(kx * x + ky * y)
    f = O.force(p, dphi)
    c = p.inv_beta_v / (p.d_p * p.dt) * a / (kx ** 2 + ky ** 2) * O.fstar_lattice(p)
    s = np.sin(kx * x + ky * y)
    assert np.abs(f[0] + c * kx * s).max() < 1e-12 * c * kx
    assert np.abs(f[1] + c * ky * s).max() < 1e-12 * c * kx


def test_force_divergence_curl_and_mean(oracle_lib):
    # T7: for a zero-mean dPhi without Nyquist content,
    #   div f = -(1/beta v) sum_I dPhi_I / (D_I dt)  (Eq. (19)),
    #   curl f = 0 (App. A), and the mean force vanishes.
    p = O.Params(nx=32, ny=16)
    rng = np.random.default_rng(4)
    dphi = np.empty((3, p.ny, p.nx))
    for s in range(3):
        spec = np.fft.fft2(rng.normal(size=(p.ny, p.nx)))
        spec[0, 0] = 0
        spec[p.ny // 2, :] = 0
        spec[:, p.nx // 2] = 0
        dphi[s] = 1e-5 * np.fft.ifft2(spec).real
    f = O.force(p, dphi) / O.fstar_lattice(p)
    div = O.spectral_op(p, f[0], 0, 1) + O.spectral_op(p, f[1], 1, 1)
    src = -(dphi[0] / p.d_p + dphi[1] / p.d_p + dphi[2] / p.d_s) / p.dt
    assert np.abs(div - src).max() < 1e-10 * np.abs(src).max()
    curl = O.spectral_op(p, f[1], 0, 1) - O.spectral_op(p, f[0], 1, 1)
    assert np.abs(curl).max() < 1e-10 * np.abs(src).max()
    assert abs(f[0].mean()) < 1e-14 * np.abs(f).max() and abs(f[1].mean()) < 1e-14 * np.abs(f).max()
