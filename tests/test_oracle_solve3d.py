"""Pins of the oracle's three-dimensional single-chain solve (the extension
named in Sec. 2 and Sec. 5; Eqs. (6)-(11) on an nz x ny x nx box)."""
import numpy as np
import pytest

import oracle as O


def test_fft3d_matches_numpy(oracle_lib):
    rng = np.random.default_rng(2)
    for shape in ((4, 6, 8), (3, 5, 2), (8, 4, 10)):
        a = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
        assert np.abs(O.fft3d(a, -1) - np.fft.fftn(a)).max() < 1e-12 * np.abs(a).sum()
        assert np.abs(O.fft3d(a, +1) - np.fft.ifftn(a) * a.size).max() < 1e-12 * np.abs(a).sum()


@pytest.mark.parametrize("rule", [0, 1])
def test_one_plane_is_the_2d_solve(oracle_lib, rule):
    # nz = 1: k_z = 0 only, the same arithmetic as the 2D solve, bit for bit
    # (under either junction rule)
    p = O.Params(nx=16, ny=8, ns=8, phi_p=0.2, f_a=0.375, junction_rule=rule)
    rng = np.random.default_rng(3)
    om = 0.2 * rng.standard_normal((3, p.ny, p.nx))
    phi3, q3 = O.solve3d(p, 1, om[:, None])
    phi2, q2 = O.solve(p, om)
    assert np.array_equal(phi3[:, 0], phi2) and np.array_equal(q3, q2)


def test_fields_along_z_are_the_2d_solve_of_the_xz_plane(oracle_lib):
    # omega(x, z), uniform in y: the 3D solve equals the 2D solve on the
    # (z, x) grid (the y axis only carries the k_y = 0 mode)
    p3 = O.Params(nx=8, ny=4, ns=6, phi_p=0.2)
    nz = 12
    rng = np.random.default_rng(4)
    oxz = 0.2 * rng.standard_normal((3, nz, p3.nx))
    om = np.repeat(oxz[:, :, None, :], p3.ny, axis=2)
    phi3, q3 = O.solve3d(p3, nz, om)
    p2 = O.Params(nx=8, ny=nz, ns=6, phi_p=0.2)
    phi2, q2 = O.solve(p2, oxz)
    for y in range(p3.ny):
        assert np.abs(phi3[:, :, y, :] - phi2).max() < 1e-14
    assert np.abs(q3 - q2).max() < 1e-15


def test_homogeneous_closed_form_3d(oracle_lib):
    p = O.Params(nx=4, ny=6, ns=10, f_a=0.3, phi_p=0.25)
    phi, q = O.solve3d(p, 8, np.full((3, 8, 6, 4), 0.37))
    fa = O.n_a(p) / p.ns
    assert np.abs(phi[0] - p.phi_p * fa).max() < 1e-15
    assert np.abs(phi[1] - p.phi_p * (1 - fa)).max() < 1e-15
    assert np.abs(phi[2] - (1 - p.phi_p)).max() < 1e-15
    assert abs(q[0] - np.exp(-p.n_seg * 0.37)) < 1e-15 and abs(q[1] - np.exp(-0.37)) < 1e-16


@pytest.mark.parametrize("f_a", [0.5, 0.882])
def test_mass_exact_3d(oracle_lib, f_a):
    p = O.Params(nx=8, ny=6, ns=8, f_a=f_a, phi_p=0.2)
    rng = np.random.default_rng(5)
    phi, _ = O.solve3d(p, 10, 0.3 * rng.standard_normal((3, 10, 6, 8)))
    fa = O.n_a(p) / p.ns
    assert abs(phi[0].mean() - p.phi_p * fa) < 1e-15
    assert abs(phi[1].mean() - p.phi_p * (1 - fa)) < 1e-15
    assert abs(phi[2].mean() - (1 - p.phi_p)) < 1e-15
