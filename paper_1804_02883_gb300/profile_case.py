"""Run a few coupled steps of a benchmark workload without timing or L2
flushes, for kernel profilers:

    python -m paper_1804_02883_gb300.profile_case --workload channel --steps 2

--workload box3d runs the coupled step on a 128 x 128 x 64 box (--time
prints CUDA-event milliseconds per step).  --workload surrogate runs the
learned surrogate's network on the benchmark batch (4 x 256 x 512): --steps
rounds of one forward pass, one forward + tangent pass and one training
step.  --exact N then runs N exact steps (Fletcher-Reeves inversion to the 1e-8
tolerance, at most 100 iterations each) after the --steps truncated ones.
"""
from __future__ import annotations

import argparse

from . import binding as B
from . import workloads as W

WORKLOADS = {
    "channel": lambda: W.channel_256x512(B.MIXED_FP32),
    "ensemble32": lambda: W.ensemble_32(B.MIXED_FP32),
    "vesicle": lambda: [W.vesicle_1024x2048(B.MIXED_FP32)],
    # the vesicle grid with a short contour (N_s = 16): the streaming passes
    # of the full-size grid with a small history, for counter captures
    "stream_short": lambda: [W.with_(W.vesicle_1024x2048(B.MIXED_FP32), ns=16)],
    "plain_small": lambda: [W.plain_small()],
    "paper150": lambda: W.paper_150(B.MIXED_FP32),
}


def box3d(steps: int, timed: bool, mixed: bool = False) -> None:
    """Coupled steps on a 128 x 128 x 64 box (N_s = 16, phi_p = 0.2, the
    reverse-Poiseuille force along x; FP64, or with mixed the FP32 solves),
    state resident on the device; with timed, CUDA-event milliseconds per
    step after one warm-up step."""
    import ctypes

    import numpy as np
    import torch

    nx, ny, nz = 128, 128, 64
    run = B.RunParams(nx=nx, ny=ny, ns=16, precision=B.MIXED_FP32 if mixed else B.PLAIN_FP64, f_a=0.5, phi_p=0.2,
                      f0=2.0, seed=7)
    rng = np.random.default_rng(7)
    w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
    om = torch.from_numpy(1e-3 * rng.uniform(-1, 1, (3, nz, ny, nx))).cuda()
    pop = torch.from_numpy(np.broadcast_to(w[:, None, None, None], (19, nz, ny, nx)).copy()).cuda()
    vel = torch.zeros((3, nz, ny, nx), dtype=torch.float64, device="cuda")
    phi, force = torch.empty_like(om), torch.empty_like(vel)
    q = torch.empty(2, dtype=torch.float64, device="cuda")
    nb = ctypes.c_size_t()
    assert B.lib().epd_step3d_workspace_bytes(ctypes.byref(run.c()), nz, ctypes.byref(nb)) == 0
    ws = torch.empty(nb.value + 256, dtype=torch.uint8, device="cuda")
    wptr = (ws.data_ptr() + 255) & ~255
    st = torch.cuda.current_stream()

    def one():
        rc = B.lib().epd_step3d(ctypes.byref(run.c()), nz, om.data_ptr(), pop.data_ptr(), vel.data_ptr(),
                                phi.data_ptr(), q.data_ptr(), force.data_ptr(), wptr, nb.value, st.cuda_stream)
        assert rc == 0, rc

    if not timed:
        for _ in range(steps):
            one()
        st.synchronize()
        return
    one()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(st)
    for _ in range(steps):
        one()
    b.record(st)
    b.synchronize()
    ms = a.elapsed_time(b) / steps
    units = nx * ny * nz * run.ns * 4
    prec = "FP32 solves" if mixed else "FP64"
    print(f"box3d {nz}x{ny}x{nx} N_s={run.ns} {prec}: {ms:.3f} ms/step, {units / (ms * 1e-3):.3e} site.contour-steps/s,"
          f" Q = {q[0].item():.12f}")


def surrogate(steps: int) -> None:
    """The surrogate network's kernels on a batch of four 256 x 512 fields
    (random init, seeded inputs of the quench's amplitude)."""
    import numpy as np
    import torch

    from . import surrogate as S

    run = B.RunParams(nx=512, ny=256, ns=64, precision=B.MIXED_FP32)
    sm = S.Surrogate(run, 4, s_in=300.0, s_out=1e-3, seed=1)
    om = torch.from_numpy(1e-3 * np.random.default_rng(0).standard_normal((4, 3, 256, 512))).cuda()
    om2 = om + 1e-6
    ph = sm.forward(om)
    for _ in range(steps):
        sm.forward(om)
        sm.tangent(om, om2)
        sm.train_step(om, ph, lr=1e-4)
    torch.cuda.synchronize()


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="channel", choices=sorted(WORKLOADS) + ["box3d", "surrogate"])
    ap.add_argument("--time", action="store_true", help="box3d: print CUDA-event ms per step")
    ap.add_argument("--mixed", action="store_true", help="box3d: FP32 single-chain solves")
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--exact", type=int, default=0, help="then this many exact steps (0: none)")
    args = ap.parse_args()
    if args.workload == "box3d":
        box3d(args.steps, args.time, args.mixed)
        print("ok")
        return
    if args.workload == "surrogate":
        surrogate(args.steps)
        print("ok")
        return
    h = B.EpdLb(WORKLOADS[args.workload]())
    h.step(args.steps)
    if args.exact > 0:
        h.set_inversion(100, 1e-8)
        h.step(args.exact)
    h.sync()
    h.close()
    print("ok")


if __name__ == "__main__":
    main()
