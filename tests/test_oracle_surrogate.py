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


def test_conv_transpose_is_adjoint():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((4, 8, 16))
    w = rng.standard_normal((5, 4, 3, 3))
    g = rng.standard_normal((5, 8, 16))
    assert abs((OS.conv(x, w) * g).sum() - (x * OS.conv_transpose(g, w)).sum()) < 1e-10


def test_conv_is_correlation_with_stated_taps():
    # a single tap W[0,0,dy+1,dx+1] = 1 picks x(r + (dy, dx))
    x = np.arange(64.0).reshape(1, 8, 8)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            w = np.zeros((1, 1, 3, 3))
            w[0, 0, dy + 1, dx + 1] = 1
            y = OS.conv(x, w)
            assert y[0, 2, 5] == x[0, 2 + dy, 5 + dx]


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
