"""Learned density surrogate: training and inference through the C ABI.

The network (3x3 convolutions of dilation 1, 2, 2, 4, channels
3 -> 32 -> 32 -> 32 -> 2, tanh, circular padding) maps the fields omega to
the polymer densities; its forward, tangent, backward and Adam kernels are
the library's (epd_sur_*).  This module only marshals arguments and holds
the parameters in torch tensors.
"""
from __future__ import annotations

import ctypes

import numpy as np

from .binding import EpdLbError, RunParams, lib

LAYERS = ((3, 32), (32, 32), (32, 32), (32, 2))


def num_params() -> int:
    return int(lib().epd_sur_num_params())


def init_params(seed: int = 0, out_scale: float = 0.1) -> np.ndarray:
    """Seeded initial parameters: W ~ N(0, 1/(9 c_in)) per layer (the last
    scaled by out_scale), b = 0; layout per layer W[co][ci][3][3], b[co]."""
    rng = np.random.default_rng(seed)
    parts = []
    for li, (ci, co) in enumerate(LAYERS):
        w = rng.standard_normal((co, ci, 3, 3)) / np.sqrt(9.0 * ci)
        if li == len(LAYERS) - 1:
            w *= out_scale
        parts += [w.ravel(), np.zeros(co)]
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == num_params()
    return p


def _ws(torch, ny, nx, batch, training, device):
    nb = ctypes.c_size_t()
    rc = lib().epd_sur_workspace_bytes(ny, nx, batch, int(training), ctypes.byref(nb))
    if rc:
        raise EpdLbError(rc, "epd_sur_workspace_bytes")
    ws = torch.empty(nb.value + 256, dtype=torch.uint8, device=device)
    return ws, (ws.data_ptr() + 255) & ~255, nb.value


class Surrogate:
    """Parameters (FP32 master copy on the device), Adam moments and scales."""

    def __init__(self, run: RunParams, batch: int, params=None, s_in: float = 100.0, s_out: float = 1e-2,
                 device: str = "cuda", seed: int = 0):
        import torch

        self.torch = torch
        self.run = run
        self.batch = batch
        self.s_in = float(s_in)
        self.s_out = float(s_out)
        p = init_params(seed) if params is None else np.asarray(params, dtype=np.float32)
        self.params = torch.from_numpy(p.copy()).to(device)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.step_count = 0
        self.stream = torch.cuda.current_stream(device)
        self._ws_f = _ws(torch, run.ny, run.nx, batch, False, device)
        self._ws_t = _ws(torch, run.ny, run.nx, batch, True, device)
        self.loss_dev = torch.zeros(1, dtype=torch.float64, device=device)

    def _c(self):
        return ctypes.byref(self.run.c())

    def forward(self, omega_dev):
        """omega [batch, 3, ny, nx] FP64 device tensor -> Phi (same shape)."""
        phi = self.torch.empty_like(omega_dev)
        _, ptr, nb = self._ws_f
        rc = lib().epd_sur_forward(self._c(), omega_dev.shape[0], self.params.data_ptr(), self.s_in, self.s_out,
                                   omega_dev.data_ptr(), phi.data_ptr(), ptr, nb, self.stream.cuda_stream)
        if rc:
            raise EpdLbError(rc, "epd_sur_forward")
        return phi

    def tangent(self, omega0_dev, omega_dev):
        """Densities at omega0 (forward) and at omega to first order in
        omega - omega0 (tangent pass): (phi0, phi), each [batch, 3, ny, nx]."""
        phi0 = self.torch.empty_like(omega0_dev)
        phi = self.torch.empty_like(omega_dev)
        _, ptr, nb = self._ws_f
        rc = lib().epd_sur_tangent(self._c(), omega0_dev.shape[0], self.params.data_ptr(), self.s_in, self.s_out,
                                   omega0_dev.data_ptr(), omega_dev.data_ptr(), phi0.data_ptr(), phi.data_ptr(), ptr, nb,
                                   self.stream.cuda_stream)
        if rc:
            raise EpdLbError(rc, "epd_sur_tangent")
        return phi0, phi

    def gradients(self, omega_dev, phi_dev):
        grad = self.torch.empty_like(self.params)
        _, ptr, nb = self._ws_t
        rc = lib().epd_sur_gradients(self._c(), omega_dev.shape[0], self.params.data_ptr(), self.s_in, self.s_out,
                                     omega_dev.data_ptr(), phi_dev.data_ptr(), grad.data_ptr(), self.loss_dev.data_ptr(),
                                     ptr, nb, self.stream.cuda_stream)
        if rc:
            raise EpdLbError(rc, "epd_sur_gradients")
        return grad, float(self.loss_dev.item())

    def train_step(self, omega_dev, phi_dev, lr: float = 1e-3) -> float:
        self.step_count += 1
        _, ptr, nb = self._ws_t
        rc = lib().epd_sur_train_step(self._c(), omega_dev.shape[0], self.params.data_ptr(), self.m.data_ptr(),
                                      self.v.data_ptr(), self.step_count, ctypes.c_float(lr), self.s_in, self.s_out,
                                      omega_dev.data_ptr(), phi_dev.data_ptr(), self.loss_dev.data_ptr(), ptr, nb,
                                      self.stream.cuda_stream)
        if rc:
            raise EpdLbError(rc, "epd_sur_train_step")
        return self.loss_dev

    def params_host(self) -> np.ndarray:
        return self.params.detach().cpu().numpy()


def scales_from(omega: np.ndarray, phi: np.ndarray) -> tuple[float, float]:
    """Input and output scales from sample fields: 1/std of the omega
    fluctuations and std of the Phi_A, Phi_B fluctuations."""
    om = omega - omega.mean(axis=(-2, -1), keepdims=True)
    ph = phi[:, :2] - phi[:, :2].mean(axis=(-2, -1), keepdims=True)
    return 1.0 / max(float(om.std()), 1e-30), max(float(ph.std()), 1e-30)
