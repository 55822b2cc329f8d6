"""The cuFFT comparison of bench.py computes the single-chain solve it is
timed against: run on the host in float64 it equals the oracle's solve."""
import importlib.util
import os

import numpy as np
import pytest
import torch

import oracle as O
from paper_1804_02883_gb300 import workloads as W
from helpers import oracle_params

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


@pytest.mark.parametrize("nx,ny,ns,f_a", [(32, 16, 8, 0.5), (16, 32, 17, 0.882), (24, 20, 12, 0.3)])
def test_cufft_solve_equals_the_oracle(oracle_lib, nx, ny, ns, f_a):
    b = _bench()
    runs = [W.with_(W.plain_small(), nx=nx, ny=ny, ns=ns, f_a=f_a, seed=s) for s in (3, 4)]
    om = np.stack([W.random_omega(ny, nx, seed=10 + k) for k in range(len(runs))])
    phi, q = b.cufft_solve(torch, torch.from_numpy(om), runs[0], torch.float64)
    for k in range(len(runs)):
        want_phi, want_q = O.solve(oracle_params(runs[0]), om[k])
        assert np.abs(phi[k].numpy() - want_phi).max() < 1e-12 * np.abs(want_phi).max()
        assert np.abs(q[k].numpy() - want_q).max() < 1e-13 * want_q.max()


def test_timing_branch_and_section(monkeypatch):
    # the CUDA-event timing branch and the section's bookkeeping, with a
    # stand-in event (no device here)
    b = _bench()

    class Ev:
        n = 0

        def __init__(self, enable_timing=False):
            Ev.n += 1
            self.t = Ev.n

        def record(self, stream=None):
            pass

        def synchronize(self):
            pass

        def elapsed_time(self, other):
            return float(other.t - self.t)

    monkeypatch.setattr(torch.cuda, "Event", Ev)
    monkeypatch.setattr(torch.Tensor, "cuda", lambda self, *a, **k: self)
    runs = [W.with_(W.plain_small(), nx=16, ny=16, ns=8, seed=s) for s in (1, 2)]

    class H:
        def get_state(self, k):
            return W.random_omega(16, 16, seed=k), None, None

    seen = {}

    def graph_stub(torch_, nchains, ny, nx, ns, flush, reps):
        seen.update(nchains=nchains, ny=ny, nx=nx, ns=ns)
        return 0.25

    monkeypatch.setattr(b, "cufft_transforms_graph", graph_stub)
    out = b.cufft_section(torch, runs, H(), 0.5, torch.zeros(4), reps=3)
    assert out["propagation_ms"] == 1.0 and out["solve_ms"] == 2.0 and out["ours_chain_ms"] == 0.5
    assert out["propagation_vs_ours"] == 2.0
    # the graph-captured transforms cover both chains of every run, N_s steps
    assert seen == {"nchains": 4, "ny": 16, "nx": 16, "ns": 8}
    assert out["transforms_only_graph_ms"] == 0.25 and out["transforms_only_vs_ours"] == 0.5
    assert b.cufft_section(torch, [runs[0], W.with_(runs[1], ns=12)], H(), 0.5, torch.zeros(4)) is None
