"""Pins of the oracle's single-chain statistics, Sec. 2, Eqs. (6)-(11).

T1 homogeneous fields (closed form), T2 exact decay of a Fourier mode, T3 the
Debye linear response (textbook RPA) with second-order convergence in ds,
T4 invariance of <g(s) g'(1-s)> along the contour, T5 exact mass, and a
brute-force dense-matrix evaluation on a 4x4 grid."""
import numpy as np
import pytest
import scipy.linalg

import oracle as O


def test_homogeneous_closed_form(oracle_lib):
    # T1: for constant fields the Laplacian factor is the identity, so
    # g(s_j) = exp(-N ds * trapezoid of omega over nodes 0..j).
    p = O.Params(nx=8, ny=16, ns=12, f_a=0.5, phi_p=0.25)
    wa_c, wb_c, ws_c = 0.31, -0.17, 0.05
    wa = np.full((p.ny, p.nx), wa_c)
    wb = np.full((p.ny, p.nx), wb_c)
    g, gp = O.propagate(p, wa, wb)
    na = O.n_a(p)
    ds = 1.0 / p.ns
    node = np.array([wa_c if j < na else wb_c for j in range(p.ns + 1)])
    for j in range(p.ns + 1):
        tz = 0.0 if j == 0 else node[0] / 2 + node[1:j].sum() + node[j] / 2
        assert np.allclose(g[j], np.exp(-p.n_seg * ds * tz), rtol=1e-13, atol=0)
    omega = np.stack([wa, wb, np.full_like(wa, ws_c)])
    phi, q = O.solve(p, omega)
    assert abs(q[0] / g[-1, 0, 0] - 1) < 1e-14
    assert abs(q[1] / np.exp(-ws_c) - 1) < 1e-14
    assert np.allclose(phi[0], p.phi_p * na / p.ns, rtol=1e-13, atol=0)
    assert np.allclose(phi[1], p.phi_p * (p.ns - na) / p.ns, rtol=1e-13, atol=0)
    assert np.allclose(phi[2], 1 - p.phi_p, rtol=1e-14, atol=0)


@pytest.mark.parametrize("mode,grid", [((3, 0), (16, 8)), ((0, 2), (16, 8)), ((1, 3), (16, 8)), ((8, 0), (16, 8)),
                                       ((0, 4), (16, 8)), ((15, 0), (30, 20)), ((2, 10), (30, 20)), ((7, 3), (30, 20))])
def test_single_fourier_mode_decay(oracle_lib, mode, grid):
    # T2: with omega = 0 each contour step multiplies a Fourier mode by
    # exp(-R_G^2 k^2 ds) exactly, so after the whole chain the amplitude is
    # eps exp(-R_G^2 k^2).  A non-square grid separates the two axes; mode
    # (8, 0) is the x-Nyquist mode of the 16-wide grid (k = pi/dx); the 30 x 20
    # grid takes the DFT of lengths that are not powers of two.
    mx, my = mode
    p = O.Params(nx=grid[0], ny=grid[1], ns=10, rg=0.7)
    x = np.arange(p.nx) * p.dx
    y = np.arange(p.ny) * p.dx
    kx = 2 * np.pi * mx / (p.nx * p.dx)
    ky = 2 * np.pi * my / (p.ny * p.dx)
    eps = 0.3
    g0 = 1 + eps * np.cos(kx * x[None, :] + ky * y[:, None])
    z = np.zeros((p.ny, p.nx))
    g, _ = O.propagate(p, z, z, g0)
    want = 1 + eps * np.exp(-p.rg ** 2 * (kx ** 2 + ky ** 2)) * np.cos(kx * x[None, :] + ky * y[:, None])
    assert np.abs(g[-1] - want).max() < 1e-14


def debye(xx):
    return 2 * (np.exp(-xx) + xx - 1) / xx ** 2


def test_debye_linear_response_second_order(oracle_lib):
    # T3: omega_A = omega_B = eps cos(k x) gives, to first order in eps,
    # Phi_P - phi_p = -phi_p N eps g_D(k^2 R_G^2) cos(k x), g_D the Debye
    # function.  The cos(kx) coefficient has no O(eps^2) part; the scheme's
    # error is O(ds^2) (symmetric splitting + trapezoid).
    eps = 1e-7
    errs = []
    for ns in (16, 32, 64, 128):
        p = O.Params(nx=32, ny=4, ns=ns, phi_p=0.3, f_a=0.5)
        x = np.arange(p.nx) * p.dx
        k = 2 * np.pi * 2 / (p.nx * p.dx)
        w = np.broadcast_to(eps * np.cos(k * x)[None, :], (p.ny, p.nx))
        omega = np.stack([w, w, np.zeros_like(w)])
        phi, _ = O.solve(p, omega)
        dphi = phi[0] + phi[1] - p.phi_p
        coef = 2 * (dphi * np.cos(k * x)[None, :]).mean()
        want = -p.phi_p * p.n_seg * eps * debye(k ** 2 * p.rg ** 2)
        errs.append(abs(coef / want - 1))
    assert errs[-1] < 2e-4
    for a, b in zip(errs[:-1], errs[1:]):
        assert 3.6 < a / b < 4.4, errs


def test_contour_split_invariance(oracle_lib):
    # T4: <g(s_j) g'(1 - s_j)>_r = Q_P for every node j (the Laplacian factor
    # is self-adjoint and each chain's half-step factors mirror the other's).
    p = O.Params(nx=16, ny=32, ns=20, f_a=0.35)
    rng = np.random.default_rng(5)
    wa = 0.2 * rng.standard_normal((p.ny, p.nx))
    wb = 0.2 * rng.standard_normal((p.ny, p.nx))
    g, gp = O.propagate(p, wa, wb)
    qp = g[-1].mean()
    for j in range(p.ns + 1):
        assert abs((g[j] * gp[p.ns - j]).mean() / qp - 1) < 1e-13
    assert abs(gp[-1].mean() / qp - 1) < 1e-13


@pytest.mark.parametrize("f_a", [0.5, 0.3, 0.0, 1.0, 0.882])
def test_mass_exact(oracle_lib, f_a):
    # T5: <Phi_A + Phi_B> = phi_p and <Phi_S> = 1 - phi_p for any fields.
    p = O.Params(nx=32, ny=16, ns=17, f_a=f_a, phi_p=0.15)
    rng = np.random.default_rng(6)
    omega = 0.3 * rng.standard_normal((3, p.ny, p.nx))
    phi, q = O.solve(p, omega)
    assert abs(phi[0].mean() + phi[1].mean() - p.phi_p) < 1e-14
    assert abs(phi[2].mean() - (1 - p.phi_p)) < 1e-14
    if f_a == 0.0:
        assert np.all(phi[0] == 0)
    if f_a == 1.0:
        assert np.all(phi[1] == 0)


def test_block_boundary_rounding(oracle_lib):
    assert O.n_a(O.Params(ns=128, f_a=0.3)) == 38
    assert O.n_a(O.Params(ns=17, f_a=0.882)) == 15
    assert O.n_a(O.Params(ns=64, f_a=0.5)) == 32


@pytest.mark.parametrize("nx,ny", [(8, 4), (10, 6)])
def test_dense_matrix_brute_force(oracle_lib, nx, ny):
    # Brute force on a 4x8 (and a 6x10) grid, N_s = 4: the Laplacian as a
    # dense matrix built from the DFT definition, exp(R_G^2 ds L) by scipy's
    # expm, the contour recursion with dense matrices, trapezoid sums.
    p = O.Params(nx=nx, ny=ny, ns=4, f_a=0.5, phi_p=0.2, rg=0.9)
    n = p.n
    rng = np.random.default_rng(8)
    omega = 0.4 * rng.standard_normal((3, p.ny, p.nx))

    def k_axis(m, nn):
        mm = m if m <= nn // 2 else m - nn
        return 2 * np.pi * mm / (nn * p.dx)

    ys, xs = np.divmod(np.arange(n), p.nx)
    lap = np.zeros((n, n))
    for my in range(p.ny):
        for mx in range(p.nx):
            kk = k_axis(mx, p.nx) ** 2 + k_axis(my, p.ny) ** 2
            ph = np.exp(2j * np.pi * (mx * xs / p.nx + my * ys / p.ny))
            lap += (-kk * np.outer(ph, ph.conj())).real / n
    ds = 1 / p.ns
    T = scipy.linalg.expm(p.rg ** 2 * ds * lap)
    na = O.n_a(p)
    wa, wb, ws = (o.ravel() for o in omega)
    fw = [wa if j < na else wb for j in range(p.ns + 1)]
    bw = [fw[p.ns - j] for j in range(p.ns + 1)]

    def chain(fields):
        g = [np.ones(n)]
        for j in range(p.ns):
            e0 = np.exp(-p.n_seg * fields[j] * ds / 2)
            e1 = np.exp(-p.n_seg * fields[j + 1] * ds / 2)
            g.append(e1 * (T @ (e0 * g[-1])))
        return g

    g, gp = chain(fw), chain(bw)
    qp = g[-1].mean()
    wA = [0.5 * ds if j in (0, na) else ds for j in range(na + 1)]
    wB = [0.5 * ds if j in (na, p.ns) else ds for j in range(na, p.ns + 1)]
    ia = sum(w * g[j] * gp[p.ns - j] for w, j in zip(wA, range(na + 1)))
    ib = sum(w * g[j] * gp[p.ns - j] for w, j in zip(wB, range(na, p.ns + 1)))
    phi, q = O.solve(p, omega)
    assert abs(q[0] / qp - 1) < 1e-13
    assert np.abs(phi[0].ravel() - p.phi_p * ia / qp).max() < 1e-13
    assert np.abs(phi[1].ravel() - p.phi_p * ib / qp).max() < 1e-13
    qs = np.exp(-ws).mean()
    assert np.abs(phi[2].ravel() - (1 - p.phi_p) * np.exp(-ws) / qs).max() < 1e-14
