"""Learned density surrogate on the GPU: forward and gradients against the
oracle's FP64 restatement (with the GPU's bfloat16 rounding points), training
on exact (omega, Phi) pairs, its gain over the trivial prediction, and the
exact-every-k controller of the time stepper."""
import numpy as np
import pytest

import paper_1804_02883_gb300 as P
from paper_1804_02883_gb300 import surrogate as S
from paper_1804_02883_gb300 import workloads as W
from oracle import surrogate as OS

pytestmark = pytest.mark.gpu


def rand_params(seed):
    rng = np.random.default_rng(seed)
    parts = []
    for ci, co in OS.LAYERS:
        parts += [rng.standard_normal(co * ci * 9) / np.sqrt(9 * ci), 0.1 * rng.standard_normal(co)]
    return np.concatenate(parts).astype(np.float32)


@pytest.fixture(scope="module")
def torch():
    import torch as t
    P.lib()
    return t


@pytest.mark.parametrize("ny,nx", [(32, 64), (64, 32), (16, 16)])
def test_forward_matches_oracle(torch, ny, nx):
    run = P.RunParams(nx=nx, ny=ny, ns=8, precision=P.MIXED_FP32, phi_p=0.2, f_a=0.5)
    p = rand_params(11)
    om = 0.01 * np.random.default_rng(ny + nx).standard_normal((2, 3, ny, nx))
    sur = S.Surrogate(run, 2, params=p, s_in=100.0, s_out=1e-3)
    phi = sur.forward(torch.from_numpy(om).cuda()).cpu().numpy()
    for b in range(2):
        want = OS.densities(p.astype(np.float64), om[b], 100.0, 1e-3, 0.2, 0.5, emulate_bf16=True)
        for c in range(2):
            spread = np.abs(want[c] - want[c].mean()).max()
            # FP32 accumulation order and tanhf vs the FP64 oracle can move a value
            # across a bfloat16 rounding boundary (relative 2^-8) here and there
            assert np.abs(phi[b, c] - want[c]).max() < 3e-3 * spread
            assert abs(phi[b, c].mean() - want[c].mean()) < 1e-15
        assert np.abs(phi[b, 2] - want[2]).max() < 1e-6 * want[2].max()


def test_gradients_match_oracle(torch):
    run = P.RunParams(nx=64, ny=32, ns=8, precision=P.MIXED_FP32, phi_p=0.2)
    p = rand_params(11)
    rng = np.random.default_rng(0)
    om = 0.01 * rng.standard_normal((2, 3, 32, 64))
    phs = np.stack([OS.densities(rand_params(12).astype(np.float64), om[b], 100.0, 1e-3, 0.2, 0.5) for b in range(2)])
    sur = S.Surrogate(run, 2, params=p, s_in=100.0, s_out=1e-3)
    g, loss = sur.gradients(torch.from_numpy(om).cuda(), torch.from_numpy(phs).cuda())
    g = g.cpu().numpy()
    lo, go = OS.loss_and_grad(p.astype(np.float64), list(om), list(phs), 100.0, 1e-3, emulate_bf16=True)
    assert abs(loss / lo - 1) < 1e-5
    assert np.linalg.norm(g - go) / np.linalg.norm(go) < 1e-3
    # element by element, per parameter tensor (weights and biases of every
    # layer): each gradient entry within 1e-3 of its tensor's largest entry.
    # Both sides round the same values to bfloat16; what remains is the FP32
    # accumulation order over the 2 x 32 x 64 pixels and tanhf, which can
    # move one activation across a bfloat16 boundary (2^-8 of one term).
    off = 0
    for li, (ci, co) in enumerate(OS.LAYERS):
        for name, size in (("w", co * ci * 9), ("b", co)):
            gt, got = g[off:off + size], go[off:off + size]
            off += size
            assert np.abs(gt - got).max() <= 1e-3 * np.abs(got).max(), (li, name)
    assert off == go.size


@pytest.mark.parametrize("ny,nx", [(32, 64), (64, 32)])
def test_tangent_matches_oracle(torch, ny, nx):
    # the density change along a small field change (the size of one
    # diffusion update) from the tangent pass, element by element against the
    # oracle's forward-mode derivative with the same bfloat16 rounding points
    run = P.RunParams(nx=nx, ny=ny, ns=8, precision=P.MIXED_FP32, phi_p=0.2, f_a=0.5)
    p = rand_params(13)
    rng = np.random.default_rng(ny * nx)
    om0 = 0.01 * rng.standard_normal((2, 3, ny, nx))
    dom = 1e-5 * rng.standard_normal((2, 3, ny, nx))
    sur = S.Surrogate(run, 2, params=p, s_in=100.0, s_out=1e-3)
    phi0, phi = sur.tangent(torch.from_numpy(om0).cuda(), torch.from_numpy(om0 + dom).cuda())
    phi0, phi = phi0.cpu().numpy(), phi.cpu().numpy()
    for b in range(2):
        want0 = OS.densities(p.astype(np.float64), om0[b], 100.0, 1e-3, 0.2, 0.5, emulate_bf16=True)
        assert np.abs(phi0[b, :2] - want0[:2]).max() < 3e-3 * np.abs(want0[:2] - want0[:2].mean()).max()
        want = OS.density_change(p.astype(np.float64), om0[b], dom[b], 100.0, 1e-3, emulate_bf16=True)
        got = phi[b, :2] - phi0[b, :2]
        # BF16 tangents (relative 2^-8 per stored value) through four layers
        assert np.abs(got - want).max() < 2e-2 * np.abs(want).max()
        assert np.corrcoef(got.ravel(), want.ravel())[0, 1] > 0.999
        # the solvent density is Eq. (11) at the new field
        es = np.exp(-(om0[b, 2] + dom[b, 2]))
        assert np.abs(phi[b, 2] - 0.8 * es / es.mean()).max() < 1e-6


def exact_pairs(torch, run, count, seed):
    """(omega, Phi) of exact single-chain solves on quench-like fields."""
    h = P.EpdLb([run])
    oms, phs = [], []
    for k in range(count):
        om = W.random_omega(run.ny, run.nx, seed=seed + k, amp=3e-3)
        phi, _ = h.solve(0, om)
        oms.append(om)
        phs.append(phi)
    h.close()
    return np.stack(oms), np.stack(phs)


def test_training_beats_the_trivial_prediction(torch):
    # what the network gains over the method without it: after training on
    # exact pairs, its densities on held-out fields are much closer to the
    # exact solve than the homogeneous prediction Phi = <Phi>
    run = P.RunParams(nx=64, ny=64, ns=16, precision=P.MIXED_FP32, phi_p=0.2, f_a=0.5)
    om, ph = exact_pairs(torch, run, 40, seed=100)
    ot, pt = exact_pairs(torch, run, 8, seed=900)
    s_in, s_out = S.scales_from(om, ph)
    sur = S.Surrogate(run, 8, s_in=s_in, s_out=s_out, seed=3)
    om_d, ph_d = torch.from_numpy(om).cuda(), torch.from_numpy(ph).cuda()
    first = None
    for it in range(400):
        k = (it * 8) % 40
        idx = torch.arange(k, k + 8) % 40
        loss = float(sur.train_step(om_d[idx], ph_d[idx], lr=3e-3).item())
        first = loss if first is None else first
    assert loss < 0.2 * first
    pred = sur.forward(torch.from_numpy(ot).cuda()).cpu().numpy()
    res = np.sqrt(((pred[:, :2] - pt[:, :2]) ** 2).mean())
    trivial = np.sqrt(((pt[:, :2] - pt[:, :2].mean(axis=(2, 3), keepdims=True)) ** 2).mean())
    assert res < 0.5 * trivial, (res, trivial)


def test_controller_exact_every_k(torch):
    run = W.with_(W.plain_small(), precision=P.MIXED_FP32, f0=0.0)
    h = P.EpdLb([run])
    params = S.init_params(seed=1, out_scale=0.0)  # predicts the exact means
    # the residual is relative to the exact density fluctuations: a network
    # that predicts only the exact means has residual 1
    h.set_surrogate(params, s_in=300.0, s_out=1e-3, exact_every=8, residual_tol=2.0)
    h.step(24)
    st = h.surrogate_stats()
    assert st["steps"] == 24 and st["exact"] == 3 and st["surrogate"] == 21 and st["forced_exact"] == 0
    assert abs(st["last_residual"] - 1.0) < 1e-6
    ob = h.observables(0)
    assert abs((ob["mean_phi_a"] + ob["mean_phi_b"]) / run.phi_p - 1) < 1e-12
    # a network that misses the fluctuations fails a tolerance below 1: the
    # fallback fires and the steps stay exact
    h.set_surrogate(params, s_in=300.0, s_out=1e-3, exact_every=8, residual_tol=0.5)
    h.step(10)
    st = h.surrogate_stats()
    assert st["forced_exact"] > 0 and st["falling_back"] == 1 and st["surrogate"] == 0
    # a residual tolerance that cannot be met forces exact steps
    h.set_surrogate(params, s_in=300.0, s_out=1e-3, exact_every=8, residual_tol=0.0)
    h.step(5)
    st = h.surrogate_stats()
    assert st["exact"] == 5 and st["surrogate"] == 0 and st["forced_exact"] == 4 and st["falling_back"] == 1
    h.set_surrogate(None, 0, 0, exact_every=0)
    h.step(2)
    h.close()


def test_hold_force_keeps_the_exact_force_on_surrogate_steps(torch):
    # Step 1 is exact in both handles; on step 2 (a surrogate step) both take
    # the same surrogate densities, but the LB sees the surrogate's own force
    # in one handle and the held force of step 1 in the other.  The collision
    # velocity is (j + f/2)/rho with the same j and rho, so the two differ by
    # half the force difference, and repeating the held step reproduces it.
    run = W.with_(W.plain_small(), precision=P.MIXED_FP32, f0=0.0, noise_amp=1e-2)
    params = S.init_params(seed=2, out_scale=0.05)
    hs = [P.EpdLb([run]) for _ in range(3)]
    hs[0].set_surrogate(params, s_in=300.0, s_out=1e-3, exact_every=100, residual_tol=1e9, hold_force=False)
    hs[1].set_surrogate(params, s_in=300.0, s_out=1e-3, exact_every=100, residual_tol=1e9, hold_force=True)
    hs[2].set_surrogate(params, s_in=300.0, s_out=1e-3, exact_every=100, residual_tol=1e9, hold_force=True)
    for h in hs:
        h.step(2)
    own, held, held2 = (h.velocity(0) for h in hs)
    pa, pb = hs[0].densities(0)[0], hs[1].densities(0)[0]
    assert np.array_equal(pa, pb)  # the densities do not depend on the force choice
    assert np.array_equal(held, held2)
    assert np.abs(own - held).max() > 1e-3 * np.abs(held).max()
    for h in hs:
        st = h.surrogate_stats()
        assert st["exact"] == 1 and st["surrogate"] == 1
        h.close()


def test_repeated_calls_are_bitwise_identical(torch):
    # the means inside the network passes are one-launch reductions whose
    # last block adds the partials in a fixed order (a self-resetting
    # counter): calls on the same inputs give the same bits, forward and
    # tangent, on the same workspace and on a fresh one
    run = P.RunParams(nx=64, ny=32, ns=8, precision=P.MIXED_FP32, phi_p=0.2, f_a=0.5)
    p = rand_params(23)
    rng = np.random.default_rng(5)
    om0 = torch.from_numpy(0.01 * rng.standard_normal((3, 3, 32, 64))).cuda()
    om = om0 + torch.from_numpy(1e-4 * rng.standard_normal((3, 3, 32, 64))).cuda()
    a = S.Surrogate(run, 3, params=p, s_in=100.0, s_out=1e-3)
    b = S.Surrogate(run, 3, params=p, s_in=100.0, s_out=1e-3)
    f1 = a.forward(om0).cpu().numpy()
    f2 = a.forward(om0).cpu().numpy()
    f3 = b.forward(om0).cpu().numpy()
    assert np.array_equal(f1, f2) and np.array_equal(f1, f3)
    t1 = [x.cpu().numpy() for x in a.tangent(om0, om)]
    t2 = [x.cpu().numpy() for x in a.tangent(om0, om)]
    t3 = [x.cpu().numpy() for x in b.tangent(om0, om)]
    for x, y, z in zip(t1, t2, t3):
        assert np.array_equal(x, y) and np.array_equal(x, z)
