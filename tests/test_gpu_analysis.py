"""GPU analysis of the polymer distribution against the oracle: particles
(connected clusters with Phi_P >= 0.5, labels bit for bit, gyration tensors
of Eqs. (27)-(29)), the channel width Y_2^P of Eq. (30) and sigma_Delta of
Eq. (22), on fields with particles (one across both periodic boundaries)
and on the benchmark batch."""
import numpy as np
import pytest

import oracle as O
import paper_1804_02883_gb300 as P
from paper_1804_02883_gb300 import workloads as W
from helpers import oracle_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build(oracle_lib):
    P.lib()


def _wells(ny, nx, depth):
    """omega_A = omega_B = minus a sum of Gaussian wells (one elongated, one
    across both periodic boundaries): the polymer gathers in them."""
    x = np.arange(nx)[None, :]
    y = np.arange(ny)[:, None]

    def g(cx, cy, rx, ry):
        ddx = (x - cx + nx / 2) % nx - nx / 2
        ddy = (y - cy + ny / 2) % ny - ny / 2
        return np.exp(-(ddx ** 2 / (2 * rx * rx) + ddy ** 2 / (2 * ry * ry)))

    w = -depth * (g(nx * 0.16, ny * 0.19, 3, 3) + g(nx * 0.62, ny * 0.31, 6, 2.5) + g(nx - 2, ny - 2, 3, 3.5)
                  + g(nx * 0.47, ny * 0.78, 2.5, 2.5) + g(nx * 0.81, ny * 0.62, 3, 4.5))
    return np.stack([w, w, np.zeros_like(w)])


@pytest.mark.parametrize("prec,ny,nx", [(P.PLAIN_FP64, 64, 64), (P.MIXED_FP32, 64, 64), (P.PLAIN_FP64, 32, 128),
                                      (P.PLAIN_FP64, 150, 150), (P.MIXED_FP32, 60, 90)])
def test_particles_match_the_oracle(prec, ny, nx):
    r = P.RunParams(nx=nx, ny=ny, ns=8, precision=prec, f_a=0.5, phi_p=0.2, f0=0.0)
    om = _wells(ny, nx, 0.3)
    p = oracle_params(r)
    phi, _ = O.solve(p, om)
    php = phi[0] + phi[1]
    # thresholding is decided in the precision of each side: keep a margin
    assert np.abs(php - 0.5).min() > 1e-4
    olab, ost, ocnt = O.particles(p, phi)
    assert ocnt == 5
    h = P.EpdLb([r])
    h.set_state(0, om, None, None)
    cnt, st, lab = h.particles(0, 0.5, labels=True)
    assert cnt == ocnt and np.array_equal(lab, olab)
    tol = 1e-12 if prec == P.PLAIN_FP64 else 2e-5
    assert np.array_equal(st[:, 0], ost[:, 0])
    # G_xy and c vanish for round, axis-aligned particles: their scale is the
    # tensor's (G_xx, G_yy); c_rel is at most 1
    tensor = max(np.abs(ost[:, 4]).max(), np.abs(ost[:, 6]).max())
    for j, name in enumerate(P.EpdLb.PARTICLE_FIELDS[1:], start=1):
        scale = tensor if name in ("gxy", "c") else 1.0 if name == "c_rel" else np.abs(ost[:, j]).max()
        assert np.abs(st[:, j] - ost[:, j]).max() <= tol * scale, name
    assert ost[:, 9].max() > 0.1  # an elongated particle: c_rel well above 0
    # the width of the same fields: exact on the GPU's own densities, within
    # the solve's parity on the oracle's
    gphi, _ = h.densities(0)
    assert abs(h.width(0) - O.width(p, gphi)) < 1e-13
    assert abs(h.width(0) - O.width(p, phi)) < (1e-11 if prec == P.PLAIN_FP64 else 1e-6)
    h.close()


def test_particles_limits_and_errors():
    r = P.RunParams(nx=64, ny=64, ns=8, precision=P.PLAIN_FP64, f_a=0.5, phi_p=0.2, f0=0.0)
    h = P.EpdLb([r])
    h.set_state(0, _wells(64, 64, 0.3), None, None)
    cnt, st, _ = h.particles(0, 0.5, max_particles=2)
    assert cnt == 5 and st.shape == (2, 10)
    cnt0, _, lab = h.particles(0, 1e9, labels=True)  # nothing above the threshold
    assert cnt0 == 0 and (lab == -1).all()
    with pytest.raises(P.EpdLbError):
        h.particles(0, 0.0)
    h.close()


def test_width_and_sigma_delta_on_the_benchmark_batch():
    # four 256 x 512 runs after a few steps: no particles yet (incubation),
    # width near 1, and the GPU's values equal the oracle's on the GPU's own
    # densities
    runs = W.channel_256x512(P.MIXED_FP32)
    h = P.EpdLb(runs)
    h.step(3)
    h.sync()
    p = oracle_params(runs[0])
    phis = [h.densities(k)[0] for k in range(len(runs))]
    for k in range(len(runs)):
        assert abs(h.width(k) - O.width(p, phis[k])) < 1e-13
        assert abs(h.width(k) - 1.0) < 1e-2
        assert h.particles(k, 0.5)[0] == 0
    for a, b in ((0, 1), (1, 3), (2, 2)):
        assert abs(h.sigma_delta(a, b) - O.sigma_delta(p, phis[a], phis[b])) <= 1e-13 * max(1e-30, O.sigma_delta(p, phis[a], phis[b])) + 1e-18
    h.close()


def test_sigma_delta_coupled_against_uncoupled():
    # the paper's use: the same initial state with and without the LB
    # coupling (1/(beta v) = 0); the runs sit in two groups of one handle
    base = P.RunParams(nx=64, ny=64, ns=8, precision=P.PLAIN_FP64, f_a=0.5, phi_p=0.2, f0=2.0, noise_amp=0.05, seed=3)
    runs = [base, W.with_(base, inv_beta_v=0.0)]
    h = P.EpdLb(runs)
    h.step(3)
    h.sync()
    p0, p1 = oracle_params(runs[0]), oracle_params(runs[1])
    s0, s1 = O.initial_state(p0), O.initial_state(p1)
    O.step(p0, s0, 3)
    O.step(p1, s1, 3)
    want = O.sigma_delta(p0, s0.phi, s1.phi)
    got = h.sigma_delta(0, 1)
    assert want > 0 and abs(got - want) <= 1e-8 * want
    h.close()


def test_observables_and_reruns_on_the_benchmark_batch():
    # the two-stage reductions: the means, sigma of Eq. (21) and max |u| equal
    # plain sums over the GPU's own fields, and a rerun of each reduction is
    # bitwise equal
    runs = W.channel_256x512(P.MIXED_FP32)
    h = P.EpdLb(runs)
    h.step(3)
    h.sync()
    p = oracle_params(runs[1])
    phi, _ = h.densities(1)
    vel = h.velocity(1)
    ob = h.observables(1)
    for k, key in enumerate(("mean_phi_a", "mean_phi_b", "mean_phi_s")):
        assert abs(ob[key] - phi[k].mean()) < 1e-14
    s = O.sigma(p, phi)
    assert s > 0 and abs(ob["sigma"] - s) <= 1e-13 * s
    vmax = np.sqrt(vel[0] ** 2 + vel[1] ** 2).max()
    assert vmax > 0 and abs(ob["max_u"] - vmax) <= 1e-15 * vmax
    assert abs(ob["lb_mass"] - 1) < 1e-6
    assert ob == h.observables(1)
    assert h.width(2) == h.width(2)
    assert h.sigma_delta(0, 3) == h.sigma_delta(0, 3)
    h.close()
