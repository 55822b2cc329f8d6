"""Pins of the oracle's FFT (T6): radix-2 transform (and the tabulated DFT of
lengths that are not powers of two, such as the paper's 150-site axes)
against the O(n^2) DFT summed in long double, and the 2D transform against a
direct double sum."""
import numpy as np
import pytest


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 32, 64, 128, 256, 512, 1024, 2048, 3, 5, 6, 10, 12, 30, 150, 240])
@pytest.mark.parametrize("sign", [-1, 1])
def test_fft1d_matches_naive_dft(oracle_lib, n, sign):
    rng = np.random.default_rng(n + 7 * (sign + 1))
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    got = oracle_lib.fft1d(x, sign)
    ref = oracle_lib.dft_naive(x, sign)
    scale = np.abs(ref).max()
    # the tabulated DFT of other lengths sums n terms per output
    bound = max(1, np.log2(n)) if n & (n - 1) == 0 else np.sqrt(n)
    assert np.abs(got - ref).max() <= 2e-15 * bound * scale * 4


@pytest.mark.parametrize("ny,nx", [(8, 16), (6, 10)])
def test_fft2d_matches_direct_sum(oracle_lib, ny, nx):
    rng = np.random.default_rng(3)
    a = rng.standard_normal((ny, nx)) + 1j * rng.standard_normal((ny, nx))
    ky = np.arange(ny)[:, None, None, None]
    kx = np.arange(nx)[None, :, None, None]
    yy = np.arange(ny)[None, None, :, None]
    xx = np.arange(nx)[None, None, None, :]
    kern = np.exp(-2j * np.pi * (ky * yy / ny + kx * xx / nx))
    ref = (kern * a[None, None]).sum(axis=(2, 3))
    got = oracle_lib.fft2d(a, -1)
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()


def test_fft2d_round_trip(oracle_lib):
    rng = np.random.default_rng(4)
    a = rng.standard_normal((32, 64)) + 1j * rng.standard_normal((32, 64))
    back = oracle_lib.fft2d(oracle_lib.fft2d(a, -1), +1) / a.size
    assert np.abs(back - a).max() < 1e-14 * 16
