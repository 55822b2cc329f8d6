"""Workload presets and seeded input generators.

Shared by the tests, the benchmark and the CPU-baseline leg; holds no part of
the method's arithmetic (parameters and random inputs only).

The paper measures on no public dataset: its workload is the synthetic quench
of Sec. 3 (homogeneous fields plus a small random noise) on a periodic grid,
which the presets below reproduce at the sizes of the benchmark
configurations.  Forces f0 are in units of f* = rho R_G / tau^2, the unit in
which the paper quotes every force (Sec. 4).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from .binding import MIXED_FP32, PLAIN_FP64, RunParams


def plain_small(seed: int = 1) -> RunParams:
    """64x64 grid, AB diblock f_A = 0.5 in solvent, polymer fraction 0.3,
    N_s = 32, +-1e-3 noise, chi_BS = 0.75, LB gamma = 0 (tau = 1),
    reverse-Poiseuille force 1e-6; FP64 throughout."""
    return RunParams(nx=64, ny=64, ns=32, precision=PLAIN_FP64, f_a=0.5, phi_p=0.3, f0=1e-6,
                     noise_amp=1e-3, seed=seed)


SHEAR_AMPLITUDES = (0.0, 1e-6, 4e-6, 1.6e-5)


def channel_256x512(precision: int = MIXED_FP32, seed: int = 2) -> list[RunParams]:
    """256 x 512 periodic grid (flow along the 512-site axis, force sign
    flipped at mid-channel), N_s = 64, polymer fraction 0.2, +-1e-3 noise, one
    run per shear amplitude 0, 1e-6, 4e-6, 1.6e-5."""
    return [RunParams(nx=512, ny=256, ns=64, precision=precision, f_a=0.5, phi_p=0.2, f0=f,
                      noise_amp=1e-3, seed=seed + 1000 * k) for k, f in enumerate(SHEAR_AMPLITUDES)]


def ensemble_32(precision: int = MIXED_FP32) -> list[RunParams]:
    """32 independent runs: 8 each of 128x128, 256x128, 256x512, 512x256
    (ny x nx; the flow axis is x), N_s cycling 32, 64, 96, 128, shear
    amplitudes log-spaced 1e-7..1e-5, seeds 100 + k."""
    shapes = [(128, 128), (256, 128), (256, 512), (512, 256)]
    nss = [32, 64, 96, 128]
    runs = []
    for k in range(32):
        ny, nx = shapes[k % 4]
        f0 = 1e-7 * 100.0 ** (k / 31.0)
        runs.append(RunParams(nx=nx, ny=ny, ns=nss[(k // 4) % 4], precision=precision, f_a=0.5, phi_p=0.2,
                              f0=f0, noise_amp=1e-3, seed=100 + k))
    return runs


def vesicle_1024x2048(precision: int = MIXED_FP32, seed: int = 4, f0: float = 8e-6) -> RunParams:
    """1024 x 2048 grid, asymmetric diblock f_A = 0.3, polymer fraction 0.15,
    N_s = 128, +-1e-3 noise, chi_BS = -0.15 (vesicle systems, Sec. 3)."""
    return RunParams(nx=2048, ny=1024, ns=128, precision=precision, f_a=0.3, phi_p=0.15, chi_bs=-0.15,
                     f0=f0, noise_amp=1e-3, seed=seed)


def paper_150(precision: int = MIXED_FP32, runs: int = 64, seed: int = 200) -> list[RunParams]:
    """The paper's own system (Sec. 3, Sec. 4): 50 R_G x 50 R_G boxes of
    150 x 150 sites, N = N_s = 17, q_A = 0.882 (15 of 17 contour intervals A),
    polymer fraction 0.1, kappa_H = 1.176, chi_AB = 1.05, chi_AS = 1.20;
    half droplet systems (chi_BS = 0.75), half vesicle systems
    (chi_BS = -0.15), reverse-Poiseuille amplitudes log-spaced over the
    paper's range 1e-5 ... 1e-3 f*, seeded +-1e-3 noise: an ensemble as the
    paper averages over."""
    out = []
    half = runs // 2
    for k in range(runs):
        f0 = 1e-5 * 100.0 ** ((k % half) / max(1, half - 1))
        out.append(RunParams(nx=150, ny=150, ns=17, precision=precision, f_a=0.882, phi_p=0.1,
                             chi_bs=0.75 if k < half else -0.15, f0=f0, noise_amp=1e-3, seed=seed + k))
    return out


def with_(p: RunParams, **kw) -> RunParams:
    return dataclasses.replace(p, **kw)


# --- seeded random inputs ---------------------------------------------------

def random_omega(ny: int, nx: int, seed: int, amp: float = 0.1) -> np.ndarray:
    """Fields omega_{A,B,S} (3, ny, nx): smooth random perturbations of
    amplitude ~amp plus white noise of amplitude amp/10."""
    rng = np.random.default_rng(seed)
    y = np.arange(ny)[:, None] / ny
    x = np.arange(nx)[None, :] / nx
    out = np.empty((3, ny, nx))
    for s in range(3):
        f = np.zeros((ny, nx))
        for _ in range(4):
            kx, ky = rng.integers(0, 4, size=2)
            f += rng.normal() * np.cos(2 * np.pi * (kx * x + ky * y) + rng.uniform(0, 2 * np.pi))
        out[s] = amp * (f / 2 + 0.1 * rng.standard_normal((ny, nx)))
    return out


def random_populations(ny: int, nx: int, seed: int, amp: float = 1e-3) -> np.ndarray:
    """Pre-collision D2Q9 populations (9, ny, nx) near rest: the rest weights
    times (1 + amp * N(0, 1))."""
    rng = np.random.default_rng(seed)
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    return w[:, None, None] * (1 + amp * rng.standard_normal((9, ny, nx)))


def random_velocity(ny: int, nx: int, seed: int, amp: float = 1e-2) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return amp * rng.standard_normal((2, ny, nx))
