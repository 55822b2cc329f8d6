"""FP64 CPU restatement of the density surrogate network -- TEST
INFRASTRUCTURE ONLY (never imported by the product).

Forward and backward of the network
    x0 = s_in (omega_c - <omega_c>)
    y_l = tanh(W_l *_{d_l} y_{l-1} + b_l), l = 1..3;  y_4 = W_4 *_{d_4} y_3 + b_4
    Phi_c = <Phi_c> + s_out (y_4,c - <y_4,c>) (c = A, B), Phi_S exact (Eq. (11))
with 3x3 kernels of dilation d_l (DILATIONS) and circular padding:
(W *_d x)[co](r) = sum_ci sum_{dy,dx} W[co, ci, dy+1, dx+1] x[ci](r + d (dy, dx)).
The tangent (jvp) is the directional derivative of the forward map along a
field change domega: dx0 = s_in (domega_c - <domega_c>),
dy_l = (1 - y_l^2) (W_l *_{d_l} dy_{l-1}), dy_4 = W_4 *_{d_4} dy_3, and
dPhi_c = s_out (dy_4,c - <dy_4,c>).  Written with numpy shifts (np.roll)
for clarity.  With bf16=True the values the GPU feeds its tensor cores --
weights, inputs, activations, tangents and output gradients -- are rounded
to bfloat16 (round to nearest even) at the same points; everything else stays
FP64.
"""
from __future__ import annotations

import numpy as np

LAYERS = ((3, 32), (32, 32), (32, 32), (32, 2))
# dilation of each layer's 3x3 kernel: the receptive field is +-9 sites
# (1 + 2 + 2 + 4), every offset in it reachable
DILATIONS = (1, 2, 2, 4)


def bf16(a) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    a32 = np.asarray(a, dtype=np.float32)
    u = a32.view(np.uint32).astype(np.uint64)
    rounded = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(params: np.ndarray):
    p = np.asarray(params, dtype=np.float64)
    out, off = [], 0
    for ci, co in LAYERS:
        w = p[off:off + co * ci * 9].reshape(co, ci, 3, 3)
        off += co * ci * 9
        b = p[off:off + co]
        off += co
        out.append((w, b))
    assert off == p.size
    return out


def _shift(x: np.ndarray, oy: int, ox: int) -> np.ndarray:
    """xs(r) = x(r + (oy, ox)), periodic."""
    return np.roll(np.roll(x, -oy, axis=1), -ox, axis=2)


def conv(x: np.ndarray, w: np.ndarray, d: int = 1) -> np.ndarray:
    """Circular 3x3 correlation of dilation d: x [ci, ny, nx], w [co, ci, 3, 3] -> [co, ny, nx]."""
    out = np.zeros((w.shape[0],) + x.shape[1:])
    for dy in range(3):
        for dx in range(3):
            out += np.einsum("oc,cyx->oyx", w[:, :, dy, dx], _shift(x, d * (dy - 1), d * (dx - 1)))
    return out


def conv_transpose(g: np.ndarray, w: np.ndarray, d: int = 1) -> np.ndarray:
    """Adjoint of conv: g [co, ny, nx] -> [ci, ny, nx]."""
    out = np.zeros((w.shape[1],) + g.shape[1:])
    for dy in range(3):
        for dx in range(3):
            t = np.einsum("oc,oyx->cyx", w[:, :, dy, dx], g)
            out += _shift(t, -d * (dy - 1), -d * (dx - 1))
    return out


def conv_weight_grad(x: np.ndarray, g: np.ndarray, d: int = 1) -> np.ndarray:
    dw = np.zeros((g.shape[0], x.shape[0], 3, 3))
    for dy in range(3):
        for dx in range(3):
            dw[:, :, dy, dx] = np.einsum("oyx,cyx->oc", g, _shift(x, d * (dy - 1), d * (dx - 1)))
    return dw


def forward(params, omega, s_in, s_out, emulate_bf16=False):
    """omega [3, ny, nx] -> (y4 [2, ny, nx], cache)."""
    r = bf16 if emulate_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    layers = unpack(params)
    x = r(s_in * (omega - omega.mean(axis=(1, 2), keepdims=True)))
    acts = [x]
    ys_f = []
    for li, (w, b) in enumerate(layers):
        z = conv(acts[-1], r(w), DILATIONS[li]) + b[:, None, None]
        if li < len(layers) - 1:
            y = np.tanh(z)
            ys_f.append(y)
            acts.append(r(y))
        else:
            acts.append(z)
    return acts[-1], (acts, ys_f)


def jvp(params, omega, domega, s_in, emulate_bf16=False):
    """Directional derivative of y4 at omega along domega: dy4 [2, ny, nx].
    The tanh derivative 1 - y^2 uses the activations as the GPU stores them
    (bfloat16 when emulated)."""
    r = bf16 if emulate_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    layers = unpack(params)
    _, (acts, _) = forward(params, omega, s_in, 1.0, emulate_bf16)
    t = r(s_in * (domega - domega.mean(axis=(1, 2), keepdims=True)))
    for li, (w, _) in enumerate(layers):
        z = conv(t, r(w), DILATIONS[li])
        if li < len(layers) - 1:
            t = r(z * (1.0 - acts[li + 1] ** 2))
        else:
            t = z
    return t


def densities(params, omega, s_in, s_out, phi_p, frac_a, emulate_bf16=False):
    """Phi [3, ny, nx] of the surrogate; frac_a = N_A / N_s."""
    y4, _ = forward(params, omega, s_in, s_out, emulate_bf16)
    phi = np.empty_like(omega)
    means = (phi_p * frac_a, phi_p * (1 - frac_a))
    for c in range(2):
        phi[c] = means[c] + s_out * (y4[c] - y4[c].mean())
    es = np.exp(-omega[2])
    phi[2] = (1 - phi_p) * es / es.mean()
    return phi


def density_change(params, omega, domega, s_in, s_out, emulate_bf16=False):
    """The surrogate's Phi_A, Phi_B change [2, ny, nx] for a field change
    domega at omega (first order, jvp)."""
    dy4 = jvp(params, omega, domega, s_in, emulate_bf16)
    return s_out * (dy4 - dy4.mean(axis=(1, 2), keepdims=True))


def loss_and_grad(params, omegas, phis, s_in, s_out, emulate_bf16=False):
    """Mean squared error of y4 against (Phi_c - <Phi_c>)/s_out over the batch,
    the A, B channels and the sites, and its gradient (flat, params layout)."""
    r = bf16 if emulate_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    layers = unpack(params)
    grads = [(np.zeros_like(w), np.zeros_like(b)) for w, b in layers]
    nb = len(omegas)
    cnt = 2 * omegas[0][0].size * nb
    loss = 0.0
    for om, ph in zip(omegas, phis):
        y4, (acts, ys_f) = forward(params, om, s_in, s_out, emulate_bf16)
        t = (ph[:2] - ph[:2].mean(axis=(1, 2), keepdims=True)) / s_out
        d = y4 - t
        loss += float((d * d).sum())
        g = r(2.0 * d / cnt)
        for li in range(len(layers) - 1, -1, -1):
            w, _ = layers[li]
            gw, gb = grads[li]
            gw += conv_weight_grad(acts[li], g, DILATIONS[li])
            gb += g.sum(axis=(1, 2))
            if li > 0:
                gx = conv_transpose(g, r(w), DILATIONS[li])
                g = r(gx * (1 - ys_f[li - 1] ** 2))
    flat = np.concatenate([np.concatenate([gw.ravel(), gb]) for gw, gb in grads])
    return loss / cnt, flat
