"""Pins of the oracle's coupled step on a 3D box: spectral derivatives on
Fourier modes, the 3D force's divergence and curl (App. A in 3D), and the
step against the 2D step for fields uniform in z, exact masses and a
stationary homogeneous state."""
import numpy as np

import oracle as O


def _grid(p, nz):
    x = (np.arange(p.nx) * p.dx)[None, None, :]
    y = (np.arange(p.ny) * p.dx)[None, :, None]
    z = (np.arange(nz) * p.dx)[:, None, None]
    return x, y, z


def test_spectral_derivatives_3d(oracle_lib):
    p = O.Params(nx=8, ny=6, ns=4)
    nz = 10
    x, y, z = _grid(p, nz)
    kx, ky, kz = 2 * np.pi * 3 / (8 * p.dx), 2 * np.pi * 1 / (6 * p.dx), 2 * np.pi * 2 / (10 * p.dx)
    f = np.cos(kx * x + ky * y + kz * z)
    s = np.sin(kx * x + ky * y + kz * z)
    for op, k in enumerate((kx, ky, kz)):
        assert np.abs(O.spectral_op3d(p, nz, f, op) + k * s).max() < 1e-12
    assert np.abs(O.spectral_op3d(p, nz, f, 3) + (kx * kx + ky * ky + kz * kz) * f).max() < 1e-11
    # the Nyquist mode along z: dropped by d/dz, kept by the Laplacian
    kn = np.pi / p.dx
    g = np.cos(kn * z) + 0 * x + 0 * y
    assert np.abs(O.spectral_op3d(p, nz, g, 2)).max() < 1e-12
    assert np.abs(O.spectral_op3d(p, nz, g, 3) + kn * kn * g).max() < 1e-10


def test_force3d_divergence_and_curl(oracle_lib):
    # div f = -(fstar/(beta v)) sum_I dPhi_I / (D_I dt) minus its mean, curl f = 0,
    # for fields without Nyquist content along any axis
    p = O.Params(nx=8, ny=8, ns=4)
    nz = 8
    rng = np.random.default_rng(3)
    raw = rng.standard_normal((3, nz, p.ny, p.nx))
    # remove the Nyquist planes so that the first derivatives are exact
    spec = np.fft.fftn(raw, axes=(1, 2, 3))
    spec[:, nz // 2] = 0
    spec[:, :, p.ny // 2] = 0
    spec[:, :, :, p.nx // 2] = 0
    dphi = 1e-3 * np.real(np.fft.ifftn(spec, axes=(1, 2, 3)))
    f = O.force3d(p, nz, dphi)
    div = sum(O.spectral_op3d(p, nz, f[a], a) for a in range(3))
    s = dphi[0] / p.d_p + dphi[1] / p.d_p + dphi[2] / p.d_s
    want = -(p.inv_beta_v / p.dt) * O.fstar_lattice(p) * (s - s.mean())
    assert np.abs(div - want).max() < 1e-9 * np.abs(want).max()
    for a, b in ((0, 1), (0, 2), (1, 2)):
        curl = O.spectral_op3d(p, nz, f[b], a) - O.spectral_op3d(p, nz, f[a], b)
        assert np.abs(curl).max() < 1e-9 * np.abs(f).max() / p.dx


def _eq3(rho, u):
    C, W = O.D3Q19_C, O.D3Q19_W
    cu = np.einsum("ia,a...->i...", C, u)
    uu = (u * u).sum(axis=0)
    return W[:, None, None, None] * rho * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * uu)


def test_step3d_uniform_in_z_is_the_2d_epd_step(oracle_lib):
    # decoupled (1/(beta v) = 0), no body force, fluid at rest: omega follows
    # the pure EPD step, which for fields uniform in z is the 2D step
    p = O.Params(nx=8, ny=12, ns=6, phi_p=0.2, inv_beta_v=0.0, f0=0.0)
    nz = 4
    rng = np.random.default_rng(4)
    om2 = 0.05 * rng.standard_normal((3, p.ny, p.nx))
    om3 = np.repeat(om2[:, None], nz, axis=1)
    pop = _eq3(np.ones((nz, p.ny, p.nx)), np.zeros((3, nz, p.ny, p.nx)))
    vel = np.zeros((3, nz, p.ny, p.nx))
    w3, pop3, v3, phi3, q3, f3 = O.step3d(p, nz, om3, pop, vel)
    st = O.State(om2.copy(), np.zeros((9, p.ny, p.nx)), np.zeros((2, p.ny, p.nx)), None, None, None)
    st.phi, st.q = O.solve(p, om2)
    st.force = np.zeros((2, p.ny, p.nx))
    st.pop = np.array([w * np.ones((p.ny, p.nx)) for w in (4 / 9, 1 / 9, 1 / 9, 1 / 9, 1 / 9, 1 / 36, 1 / 36, 1 / 36, 1 / 36)])
    O.step(p, st)
    for zz in range(nz):
        assert np.abs(w3[:, zz] - st.omega).max() < 1e-13
        assert np.abs(phi3[:, zz] - st.phi).max() < 1e-13
    assert np.abs(v3).max() == 0.0 and np.abs(pop3 - pop).max() < 1e-16


def test_step3d_masses_and_homogeneous_state(oracle_lib):
    p = O.Params(nx=8, ny=8, ns=6, phi_p=0.2, f0=0.5)
    nz = 6
    rng = np.random.default_rng(5)
    om = 0.05 * rng.standard_normal((3, nz, p.ny, p.nx))
    pop = _eq3(np.ones((nz, p.ny, p.nx)), 0.01 * rng.standard_normal((3, nz, p.ny, p.nx)))
    vel = 0.01 * rng.standard_normal((3, nz, p.ny, p.nx))
    w, pop1, v1, phi, q, f = O.step3d(p, nz, om, pop, vel)
    na = O.n_a(p)
    assert abs(phi[0].mean() - p.phi_p * na / p.ns) < 1e-15
    assert abs(phi[2].mean() - (1 - p.phi_p)) < 1e-15
    assert abs(pop1.sum() - pop.sum()) < 1e-12
    assert np.abs(f.reshape(3, -1).sum(axis=1)).max() < 1e-12 * max(1e-30, np.abs(f).max()) * f[0].size
    # homogeneous fields at rest without body force: nothing changes
    p0 = O.Params(nx=8, ny=8, ns=6, phi_p=0.2, f0=0.0)
    om0 = np.full((3, nz, 8, 8), 0.1)
    pop0 = _eq3(np.ones((nz, 8, 8)), np.zeros((3, nz, 8, 8)))
    w0, popn, vn, phin, qn, fn = O.step3d(p0, nz, om0, pop0, np.zeros((3, nz, 8, 8)))
    assert np.abs(w0 - om0).max() < 1e-15 and np.abs(fn).max() < 1e-18 and np.abs(popn - pop0).max() < 1e-16
