"""Pins of the oracle's analysis of the polymer distribution: sigma_Delta of
Eq. (22), the channel width Y_2^P of Eq. (30), particles (connected clusters
with Phi_P >= 0.5, Sec. 4) and their gyration tensors, Eqs. (27)-(29)."""
import numpy as np

import oracle as O


def _phi(p, php):
    phi = np.zeros((3, p.ny, p.nx))
    phi[0] = php  # Phi_P carried by A alone
    phi[2] = 1.0 - php
    return phi


def test_sigma_delta(oracle_lib):
    p = O.Params(nx=8, ny=4)
    rng = np.random.default_rng(1)
    a = _phi(p, 0.2 + 0.01 * rng.standard_normal((p.ny, p.nx)))
    assert O.sigma_delta(p, a, a) == 0.0
    b = a.copy()
    sgn = np.where(rng.random((p.ny, p.nx)) < 0.5, -1.0, 1.0)
    b[1] += 3e-3 * sgn  # shift Phi_P by +-3e-3 through the B field
    assert abs(O.sigma_delta(p, a, b) - 3e-3) < 1e-17


def test_width_closed_forms(oracle_lib):
    # ny = 8: rows 0..3 form the first channel (centre between rows 1 and 2),
    # distances from the centre +-1.5, +-0.5 (x dx); sum of y_c^2 per column
    # over both channels = 4 (2.25 + 0.25) = 10 dx^2
    p = O.Params(nx=4, ny=8, phi_p=0.2)
    assert abs(O.width(p, _phi(p, np.full((p.ny, p.nx), 0.2))) - 1.0) < 1e-15
    centre = np.zeros((p.ny, p.nx))
    centre[[1, 2, 5, 6]] = 0.4  # the same polymer mass on the four central rows
    assert abs(O.width(p, _phi(p, centre)) - np.sqrt(0.2)) < 1e-15
    edge = np.zeros((p.ny, p.nx))
    edge[[0, 3, 4, 7]] = 0.4
    assert abs(O.width(p, _phi(p, edge)) - np.sqrt(1.8)) < 1e-15


def test_particles_dimer_rectangle_square(oracle_lib):
    p = O.Params(nx=32, ny=16)
    f = np.zeros((p.ny, p.nx))
    f[2, 3], f[2, 4] = 0.6, 0.9              # dimer along x
    f[8:11, 10:17] = 0.7                     # 7 x 3 rectangle
    f[3:8, 22:27] = 0.55                     # 5 x 5 square
    labels, st, cnt = O.particles(p, _phi(p, f))
    assert cnt == 3 and st.shape == (3, 10)
    d = dict(zip(O.PARTICLE_FIELDS, st[0]))
    w1, w2, dx = 0.6, 0.9, p.dx
    assert d["sites"] == 2 and abs(d["content"] - 1.5) < 1e-15
    assert abs(d["gxx"] - w1 * w2 * dx * dx / (w1 + w2) ** 2) < 1e-16 and d["gxy"] == 0 and d["gyy"] == 0
    assert abs(d["c_rel"] - 1.0) < 1e-14
    assert abs(d["cx"] - (3 + w2 / (w1 + w2)) * dx) < 1e-15 and abs(d["cy"] - 2 * dx) < 1e-15
    # first site of the square (3, 22) precedes the rectangle's (8, 10)
    sq, rect = dict(zip(O.PARTICLE_FIELDS, st[1])), dict(zip(O.PARTICLE_FIELDS, st[2]))
    assert rect["sites"] == 21 and sq["sites"] == 25
    assert abs(rect["gxx"] - (49 - 1) / 12 * dx * dx) < 1e-15 and abs(rect["gyy"] - (9 - 1) / 12 * dx * dx) < 1e-15
    assert abs(rect["gxy"]) < 1e-16
    gx, gy = 4.0, 2.0 / 3.0
    assert abs(rect["c_rel"] - ((gx - gy) / (gx + gy)) ** 2) < 1e-14
    assert abs(sq["gxx"] - sq["gyy"]) < 1e-15 and abs(sq["c_rel"]) < 1e-26
    assert abs(sq["R"] - np.sqrt(2 * 24 / 12) * dx) < 1e-15
    assert set(np.unique(labels)) == {-1, 0, 1, 2}
    assert (labels[2, 3], labels[4, 24], labels[9, 12]) == (0, 1, 2)


def test_particles_connectivity_threshold_and_periodic_wrap(oracle_lib):
    p = O.Params(nx=16, ny=16)
    f = np.zeros((p.ny, p.nx))
    for k in range(4):
        f[k, k] = 0.8                 # a diagonal: four separate one-site particles
    f[10, 5] = 0.5                    # exactly at the threshold: a particle
    f[10, 7] = 0.4999999999           # below
    blob = np.zeros((p.ny, p.nx))
    blob[6:9, 9:13] = 0.9
    blob[7, 13] = 0.6
    _, st0, c0 = O.particles(p, _phi(p, f + blob))
    assert c0 == 6 and list(st0[:, 0]) == [1, 1, 1, 1, 13, 1]
    # the blob rolled across both periodic boundaries: one particle, the same
    # shape, its centre moved by the roll
    rolled = np.roll(blob, (-7, -11), axis=(0, 1))
    labels, st, cnt = O.particles(p, _phi(p, rolled))
    assert cnt == 1 and st[0, 0] == 13
    a, b = dict(zip(O.PARTICLE_FIELDS, st0[4])), dict(zip(O.PARTICLE_FIELDS, st[0]))
    for k in ("content", "gxx", "gxy", "gyy", "R", "c", "c_rel"):
        assert abs(a[k] - b[k]) <= 1e-14 * max(1.0, abs(a[k])), k
    L = p.nx * p.dx
    assert abs((a["cx"] - 11 * p.dx) % L - b["cx"]) < 1e-12 and abs((a["cy"] - 7 * p.dx) % L - b["cy"]) < 1e-12
    assert labels[15, 15] == 0 and labels[0, 0] == 0  # wraps in x and y


def test_sigma_of_eq21(oracle_lib):
    # sigma = mean |Phi_P - phi_p|: 0 for the homogeneous state, a for a field
    # that deviates by +-a everywhere, and a / 2 when half the sites deviate
    p = O.Params(nx=8, ny=4, phi_p=0.2)
    assert O.sigma(p, _phi(p, np.full((p.ny, p.nx), 0.2))) == 0.0
    rng = np.random.default_rng(2)
    sgn = np.where(rng.random((p.ny, p.nx)) < 0.5, -1.0, 1.0)
    assert abs(O.sigma(p, _phi(p, 0.2 + 1e-3 * sgn)) - 1e-3) < 1e-17
    half = np.zeros((p.ny, p.nx))
    half[:, : p.nx // 2] = 4e-3
    assert abs(O.sigma(p, _phi(p, 0.2 + half)) - 2e-3) < 1e-17
