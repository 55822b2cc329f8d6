"""Pins of the oracle's surrogate network (test infrastructure): gradient by
finite differences, adjointness of the transposed convolution, exact means,
periodic translation equivariance, and the bfloat16 rounding helper."""
import numpy as np
import pytest

from oracle import surrogate as OS


def rand_params(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    parts = []
    for ci, co in OS.LAYERS:
        parts += [scale * rng.standard_normal(co * ci * 9) / np.sqrt(9 * ci), 0.1 * rng.standard_normal(co)]
    return np.concatenate(parts)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    p = rand_params(2)
    oms = [0.01 * rng.standard_normal((3, 8, 8)) for _ in range(2)]
    phs = [np.stack([0.1 + 1e-3 * rng.standard_normal((8, 8)), 0.1 + 1e-3 * rng.standard_normal((8, 8)),
                     np.full((8, 8), 0.8)]) for _ in range(2)]
    loss, g = OS.loss_and_grad(p, oms, phs, 100.0, 1e-3)
    idx = rng.choice(p.size, 40, replace=False)
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        num = (OS.loss_and_grad(pp, oms, phs, 100.0, 1e-3)[0] - OS.loss_and_grad(pm, oms, phs, 100.0, 1e-3)[0]) / (2 * h)
        assert abs(num - g[i]) < 1e-6 * max(1.0, abs(g[i]))


@pytest.mark.parametrize("d", [1, 2, 4])
def test_conv_transpose_is_adjoint(d):
    rng = np.random.default_rng(3)
    x = rng.standard_normal((4, 16, 32))
    w = rng.standard_normal((5, 4, 3, 3))
    g = rng.standard_normal((5, 16, 32))
    assert abs((OS.conv(x, w, d) * g).sum() - (x * OS.conv_transpose(g, w, d)).sum()) < 1e-10
    # and the weight gradient is the derivative of <conv(x, w), g> in w
    dw = OS.conv_weight_grad(x, g, d)
    e = np.zeros_like(w)
    e[2, 1, 0, 2] = 1.0
    assert abs((OS.conv(x, e, d) * g).sum() - dw[2, 1, 0, 2]) < 1e-10


@pytest.mark.parametrize("d", [1, 2, 4])
def test_conv_is_correlation_with_stated_taps(d):
    # a single tap W[0,0,dy+1,dx+1] = 1 picks x(r + d (dy, dx)), periodically
    x = np.arange(16.0 * 16).reshape(1, 16, 16)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            w = np.zeros((1, 1, 3, 3))
            w[0, 0, dy + 1, dx + 1] = 1
            y = OS.conv(x, w, d)
            assert y[0, 2, 5] == x[0, (2 + d * dy) % 16, (5 + d * dx) % 16]


def test_receptive_field_of_the_dilated_stack():
    # a unit input at one site reaches exactly the offsets |oy|, |ox| <= 9 of
    # 1 + 2 + 2 + 4 (every offset in between) through four dilated layers
    assert OS.DILATIONS == (1, 2, 2, 4)
    reach = {0}
    for d in OS.DILATIONS:
        reach = {r + d * k for r in reach for k in (-1, 0, 1)}
    assert reach == set(range(-9, 10))


def test_jvp_matches_central_differences():
    # the tangent pass is the derivative of the forward map (FP64)
    rng = np.random.default_rng(21)
    p = rand_params(22)
    om = 0.01 * rng.standard_normal((3, 16, 16))
    dom = 0.01 * rng.standard_normal((3, 16, 16))
    h = 1e-4
    plus = OS.densities(p, om + h * dom, 100.0, 1e-3, 0.2, 0.5)
    minus = OS.densities(p, om - h * dom, 100.0, 1e-3, 0.2, 0.5)
    num = (plus[:2] - minus[:2]) / (2 * h)
    ana = OS.density_change(p, om, dom, 100.0, 1e-3)
    assert np.abs(num - ana).max() < 1e-6 * np.abs(ana).max()
    # linear in the field change, blind to a constant shift of omega
    assert np.abs(OS.density_change(p, om, 3.0 * dom, 100.0, 1e-3) - 3.0 * ana).max() < 1e-12 * np.abs(ana).max()
    const = np.ones_like(dom) * np.array([0.2, -0.1, 0.3])[:, None, None]
    assert np.abs(OS.density_change(p, om, const, 100.0, 1e-3)).max() < 1e-14


def test_zero_network_gives_exact_means():
    p = np.zeros(sum(co * ci * 9 + co for ci, co in OS.LAYERS))
    om = 0.01 * np.random.default_rng(4).standard_normal((3, 8, 16))
    phi = OS.densities(p, om, 100.0, 1e-3, 0.2, 0.5)
    assert np.allclose(phi[0], 0.1) and np.allclose(phi[1], 0.1)
    assert abs(phi[2].mean() - 0.8) < 1e-15


def test_translation_equivariance():
    p = rand_params(5)
    om = 0.01 * np.random.default_rng(6).standard_normal((3, 8, 16))
    a = OS.densities(p, om, 100.0, 1e-3, 0.2, 0.5)
    b = OS.densities(p, np.roll(om, (3, -5), axis=(1, 2)), 100.0, 1e-3, 0.2, 0.5)
    assert np.abs(np.roll(a, (3, -5), axis=(1, 2)) - b).max() < 1e-14


def test_bf16_rounding():
    torch = pytest.importorskip("torch")
    v = np.random.default_rng(7).standard_normal(10000) * 10.0 ** np.random.default_rng(8).integers(-6, 6, 10000)
    v = np.concatenate([v, [1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -0.0, 65504.0]])
    want = torch.from_numpy(v.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(OS.bf16(v), want)
