#!/usr/bin/env python3
"""Throughput of the hybrid LB/EPD time step on GB300.

Workload (N = 1 per GPU): four independent 256 x 512 runs (flow along the
512-site axis), N_s = 64, polymer fraction 0.2, one per reverse-Poiseuille
amplitude 0, 1e-6, 4e-6, 1.6e-5 f*, seeded +-1e-3 noise (the paper's
synthetic quench), mixed precision (FP32 propagators and LB, FP64 fields,
contour sums, Q and EPD transforms).  One step = one coupled EPD/LB time step
of all four runs: 2 single-chain solves x 2 chains x N_s contour steps plus
the EPD update, the force and one D2Q9 collide-stream per run.

Metric: propagator site.contour-step updates/s (nx ny N_s x 2 chains x
2 solves x runs per step / time); LB MLUPS and the FP64-plain path reported
beside it.  Under torchrun every rank steps its own batch (replicas, no
collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "propagator site·contour-step updates/s + LB MLUPS, 1 GB300, vs FP64 plain"
UNIT = "site·contour-steps/s"
HBM_FALLBACK = 6800.0
# FP32 (non-tensor) units of a GB300 at its maximum SM clock
FP32_SMS, FP32_LANES, FP32_MHZ = 152, 128, 2070.0
# dram__bytes_read.sum + dram__bytes_write.sum of the 8 prop_chain<9,8,16,256,1,1>
# launches of one differential solve of the channel workload (ncu, one capture)
CHAIN_DIFF_TRAFFIC_BYTES = 391.25e6 + 7.20e6


def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """The slowest rank's value (the MAX over ranks); x itself without a
    process group."""
    if dist is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank_step: float, steps: int, world: int, seconds: float) -> float:
    """Whole-job throughput: every rank steps its own batch (replicas), so the
    job processes world x the units of one rank in the slowest rank's time."""
    return units_per_rank_step * steps * world / seconds


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK, "fallback"


WORKLOADS = {
    "channel": "4 runs of 256x512 (ny x nx), N_s=64, phi_p=0.2, f_A=0.5, shear amplitudes 0/1e-6/4e-6/1.6e-5 f*, "
               "seeded +-1e-3 noise",
    "ensemble32": "32 runs: 8 each of 128x128, 256x128, 256x512, 512x256 (ny x nx), N_s cycling 32/64/96/128, "
                  "f0 log-spaced 1e-7..1e-5 f*, phi_p=0.2, seeds 100+k",
    "vesicle": "1 run of 1024x2048 (ny x nx), f_A=0.3, phi_p=0.15, chi_BS=-0.15, N_s=128, f0=8e-6 f*",
    "paper150": "64 runs of the paper's 150x150 system (50 R_G boxes), N_s=N=17, q_A=0.882, phi_p=0.1, "
                "32 droplet (chi_BS=0.75) + 32 vesicle (chi_BS=-0.15), f0 log-spaced 1e-5..1e-3 f*, seeds 200+k",
}


def workload_runs(name, precision, rank):
    from paper_1804_02883_gb300 import workloads as W

    if name == "channel":
        return W.channel_256x512(precision, seed=2 + 7919 * rank)
    if name == "ensemble32":
        return [W.with_(r, seed=r.seed + 7919 * rank) for r in W.ensemble_32(precision)]
    if name == "paper150":
        return [W.with_(r, seed=r.seed + 7919 * rank) for r in W.paper_150(precision)]
    return [W.vesicle_1024x2048(precision, seed=4 + 7919 * rank)]


def units_per_step(runs) -> float:
    return float(sum(r.nx * r.ny * r.ns * 2 * 2 for r in runs))


def sites_per_step(runs) -> float:
    return float(sum(r.nx * r.ny for r in runs))


def launches_per_step(runs, h) -> int:
    """Kernel launches of one captured step, per group of equal runs: aux
    convection 2, diffusion 2, force 3, LB 1, plus the two solves: cluster
    path 3 + the chain launches each (factors, chain, Q partials, contour
    sums), streaming paths 2 N_s + 3 each (factors, start, N_s column and row
    passes, contour or finalize)."""
    import dataclasses

    first = {}
    for k, r in enumerate(runs):
        # runs share a group when all but f0, seed and noise amplitude agree
        key = tuple(v for f, v in dataclasses.asdict(r).items() if f not in ("f0", "seed", "noise_amp"))
        first.setdefault(key, k)
    total = 0
    for k in first.values():
        t = h.tiles(k)
        solve = 3 + t["chain_launches"] if t["path"] == 2 else 2 * runs[k].ns + 3
        total += 8 + 2 * solve
    return total


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.out.close()

    def summary(self):
        if self.proc is None or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_step_time(run, nsteps: int = 1) -> float:
    """Seconds per oracle coupled step of one run (single host thread)."""
    import oracle as O

    p = O.Params(**{k: getattr(run, k) for k in O.Params.__dataclass_fields__})
    st = O.initial_state(p)
    t0 = time.perf_counter()
    O.step(p, st, nsteps)
    return (time.perf_counter() - t0) / nsteps


def run_reference(args, budget_s: float = 150.0) -> None:
    """The oracle (plain FP64 C, one host thread) on the same workload and
    config: each step is one oracle coupled step of one run of the workload
    (cycling through its runs); steps stop once budget_s seconds have passed
    (at least one), so the whole run ends within a few minutes."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O

    O.build()
    runs = workload_runs(args.workload, 0, 0)
    for _ in range(min(args.warmup, 1)):
        oracle_step_time(min(runs, key=lambda r: r.nx * r.ny * r.ns), 1)
    t = 0.0
    units = 0.0
    done = 0
    t_start = time.perf_counter()
    for k in range(args.steps):
        if done and time.perf_counter() - t_start > budget_s:
            break
        r = runs[k % len(runs)]
        t += oracle_step_time(r, 1)
        units += r.nx * r.ny * r.ns * 4
        done += 1
    value = units / t
    sample = (f"{done} oracle coupled steps, one run of the workload each (cycling its {len(runs)} runs)"
              + ("" if done == args.steps else f"; stopped after {budget_s:.0f} s of {args.steps} requested"))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": done, "warmup": args.warmup, "ms_per_step": 1e3 * t / done,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "precision": "fp64 (the oracle, one host thread)",
                   "l2": "not applicable (host)", "parallelism": "one host thread on rank 0"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def time_steps(h, stream, steps, flush, with_kernels=False):
    import torch

    per_step, kern = [], []
    for _ in range(steps):
        with torch.cuda.stream(stream):
            flush.add_(1.0)  # write a buffer larger than L2 between timed steps
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        h.step(1)
        b.record(stream)
        b.synchronize()
        per_step.append(a.elapsed_time(b))
        if with_kernels:
            kern.append(h.kernel_times())
    return per_step, kern


def precision_errors(hm, h64, nruns, np):
    """Per run, the MIXED handle hm against the PLAIN_FP64 handle h64 after
    the same steps from the same initial state: max |dPhi| relative to
    max |Phi| and to the largest fluctuation max |Phi - <Phi>| (over the three
    species), max |du| relative to max |u|.  The FP64 path matches the FP64
    oracle to 1e-10 (parity tests), so it stands in for the oracle at the
    benchmark size."""
    phi_rel, phi_fluct, vel_rel = [], [], []
    for k in range(nruns):
        a, _ = hm.densities(k)
        b, _ = h64.densities(k)
        d = np.abs(a - b).max()
        phi_rel.append(float(d / np.abs(b).max()))
        fl = max(np.abs(b[i] - b[i].mean()).max() for i in range(b.shape[0]))
        phi_fluct.append(float(d / fl) if fl > 0 else None)
        va, vb = hm.velocity(k), h64.velocity(k)
        vs = np.abs(vb).max()
        vel_rel.append(float(np.abs(va - vb).max() / vs) if vs > 0 else None)
    return {"phi_rel": phi_rel, "phi_rel_fluctuation": phi_fluct, "velocity_rel": vel_rel,
            "reference": "the PLAIN_FP64 GPU path (parity-tested to 1e-10 of the FP64 oracle)"}


def cufft_solve(torch, omega, r, dtype, timing=False):
    """The single-chain solve of Eqs. (6)-(11) written with torch.fft (cuFFT
    on a GPU), a library comparison for the hand-written transforms and never
    the product path: omega (R, 3, ny, nx) float64 of R runs with the
    parameters of r.  Per contour step of both chains of every run (batched),
    g_{j+1} = E_{j+1} irfft2(K rfft2(E_j g_j)) with E = exp(-N omega ds / 2)
    of the node's block (g: node j; g': node N_s - j) and
    K = exp(-R_G^2 |k|^2 ds), every node state stored; then the trapezoid
    contour sums on [0, s_NA] and [s_NA, 1] (products in dtype, sums in
    float64), Q_P = <g(1)>, Phi_S from exp(-omega_S).  Returns (phi, q), and
    with timing also the CUDA-event ms of the propagation and of the whole
    solve (omega already on the device)."""
    import math

    dev = omega.device
    R, _, ny, nx = omega.shape
    ns, ds = r.ns, 1.0 / r.ns
    na = int(round(r.f_a * ns))
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)] if timing else None
    if timing:
        ev[0].record()
    kx = 2 * math.pi * torch.fft.rfftfreq(nx, d=r.dx, dtype=torch.float64, device=dev)
    ky = 2 * math.pi * torch.fft.fftfreq(ny, d=r.dx, dtype=torch.float64, device=dev)
    K = torch.exp(-r.rg ** 2 * (ky[:, None] ** 2 + kx[None, :] ** 2) * ds).to(dtype)
    e = torch.exp(-r.n_seg * omega[:, :2] * ds / 2).to(dtype)  # (R, 2, ny, nx): E_A, E_B
    ea, eb = e[:, 0], e[:, 1]

    def node_factor(j):  # (2R, ny, nx): chain g at node j, chain g' at node N_s - j
        return torch.cat((ea if j < na else eb, ea if ns - j < na else eb))

    hist = torch.empty((ns + 1, 2 * R, ny, nx), dtype=dtype, device=dev)
    hist[0].fill_(1.0)
    fac = node_factor(0)
    for j in range(ns):
        nxt = node_factor(j + 1)
        hist[j + 1] = nxt * torch.fft.irfft2(K * torch.fft.rfft2(fac * hist[j]), s=(ny, nx))
        fac = nxt
    if timing:
        ev[1].record()
    ia = torch.zeros((R, ny, nx), dtype=torch.float64, device=dev)
    ib = torch.zeros_like(ia)
    for j in range(ns + 1):
        prod = (hist[j, :R] * hist[ns - j, R:]).double()
        if na > 0 and j <= na:
            ia += (0.5 * ds if j in (0, na) else ds) * prod
        if na < ns and j >= na:
            ib += (0.5 * ds if j in (na, ns) else ds) * prod
    q_p = hist[ns, :R].double().mean(dim=(1, 2))
    bs = torch.exp(-omega[:, 2])
    q_s = bs.mean(dim=(1, 2))
    phi = torch.stack((r.phi_p * ia / q_p[:, None, None], r.phi_p * ib / q_p[:, None, None],
                       (1 - r.phi_p) * bs / q_s[:, None, None]), dim=1)
    q = torch.stack((q_p, q_s), dim=1)
    if not timing:
        return phi, q
    ev[2].record()
    ev[2].synchronize()
    return phi, q, ev[0].elapsed_time(ev[1]), ev[0].elapsed_time(ev[2])


def cufft_transforms_graph(torch, nchains, ny, nx, ns, flush, reps=5):
    """The transform work of one single-chain solve alone, with cuFFT: N_s
    forward and inverse real 2D transforms (rfft2, irfft2) of all nchains
    chains batched, captured once in a CUDA graph (no elementwise work, no
    launch gaps), FP32.  Returns the median CUDA-event ms of reps replays,
    L2 flushed before each.  A lower bound for any cuFFT-based solve of the
    same chains."""
    x = torch.randn((nchains, ny, nx), dtype=torch.float32, device="cuda")
    spec = torch.fft.rfft2(x)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):  # warm-up (cuFFT plans) outside the capture
        for _ in range(2):
            torch.fft.rfft2(x, out=spec)
            torch.fft.irfft2(spec, s=(ny, nx), out=x)
    torch.cuda.current_stream().wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for _ in range(ns):
            torch.fft.rfft2(x, out=spec)
            torch.fft.irfft2(spec, s=(ny, nx), out=x)
    ms = []
    for _ in range(reps):
        flush.add_(1.0)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        g.replay()
        b.record()
        b.synchronize()
        ms.append(a.elapsed_time(b))
    return statistics.median(ms)


def cufft_section(torch, runs, h, ours_ms, flush, reps=5):
    """cuFFT comparison on the workload: cufft_solve in FP32 on the runs'
    current fields (all runs on one grid with one parameter set but f0, seed
    and noise), L2 flushed before each of reps timed solves (median), beside
    our chain launch(es) of the step's differential solve, which propagate
    the same chains over the same contour steps (plus the differential term).
    Also the transforms alone in a captured graph (cufft_transforms_graph)."""
    r0 = runs[0]
    if any((r.nx, r.ny, r.ns, r.f_a, r.phi_p, r.chi_bs) != (r0.nx, r0.ny, r0.ns, r0.f_a, r0.phi_p, r0.chi_bs)
           for r in runs):
        return None
    om = torch.stack([torch.from_numpy(h.get_state(k)[0]) for k in range(len(runs))]).cuda()
    cufft_solve(torch, om, r0, torch.float32)
    prop, whole = [], []
    for _ in range(reps):
        flush.add_(1.0)
        _, _, a, b = cufft_solve(torch, om, r0, torch.float32, timing=True)
        prop.append(a)
        whole.append(b)
    tp, tw = statistics.median(prop), statistics.median(whole)
    tg = cufft_transforms_graph(torch, 2 * len(runs), r0.ny, r0.nx, r0.ns, flush, reps)
    return {"transforms_only_graph_ms": tg, "transforms_only_vs_ours": tg / ours_ms,
            "propagation_ms": tp, "solve_ms": tw, "ours_chain_ms": ours_ms, "propagation_vs_ours": tp / ours_ms,
            "note": "transforms_only: N_s rfft2 + irfft2 of every chain (batched), captured in one CUDA graph, no "
                    "elementwise work (a lower bound for a cuFFT solve); propagation/solve: the whole solve with "
                    "torch.fft and torch elementwise ops, eager launches; ours = the differential solve's chain "
                    "launch(es) from the step's timing probes (transforms, Fourier and node factors, state stores)"}


def analysis_section(torch, h, runs, flush, hbm, calls=20):
    """The observables (masses, sigma of Eq. (21), max |u|) and the analysis of
    Secs. 3-4 (sigma_Delta of Eq. (22) between runs 0 and 1, Y_2^P of Eq. (30),
    the particles of Phi_P >= 0.5 with their gyration tensors) on run 0 of the
    workload, each a host call that returns its result: CUDA-event time per
    call on the handle's stream (L2 flushed before each call, the result's
    device-to-host copy included), and the HBM fraction of the reductions'
    algorithmic bytes (FP64 fields read once)."""
    r0 = runs[0]
    n = r0.nx * r0.ny
    pop_bytes = 4 if r0.precision == 1 else 8
    fns = {"observables": (lambda: h.observables(0), 24 + 9 * pop_bytes + 2 * pop_bytes),
           "width": (lambda: h.width(0), 16),
           "particles": (lambda: h.particles(0, 0.5, 64), None)}
    if len(runs) > 1 and (runs[1].nx, runs[1].ny) == (r0.nx, r0.ny):
        fns["sigma_delta"] = (lambda: h.sigma_delta(0, 1), 32)
    out = {"sites": n}
    for name, (fn, bps) in fns.items():
        fn()
        ms = []
        for _ in range(calls):
            with torch.cuda.stream(h.stream):
                flush.add_(1.0)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(h.stream)
            fn()
            b.record(h.stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        t = statistics.median(ms)
        d = {"ms_per_call": t, "calls": calls}
        if bps is not None:
            gbs = bps * n / (t * 1e-3) / 1e9
            d.update({"bytes_per_site": bps, "achieved_gbs": gbs, "frac": gbs / hbm})
        out[name] = d
    out["note"] = ("two launches per reduction (a fixed grid of partial sums, then one block summing them in a "
                   "fixed order) and the copy of the result: launch- and latency-bound at this size")
    return out


def train_surrogate(P, W, torch, runs, pairs):
    """The learned density surrogate trained online on exact (omega, Phi)
    pairs streamed from the exact path of `runs`: every training step draws
    its batch from a replay pool of 1024 pairs into which the exact runs,
    advanced one step per training step and re-seeded every 1250 steps,
    write their newest pairs.  Returns (surrogate, s_in, s_out, info)."""
    from paper_1804_02883_gb300 import surrogate as S

    n_runs, (ny, nx) = len(runs), (runs[0].ny, runs[0].nx)
    pool_n, batch, reseed = 1024, 4, 1250
    om = torch.empty((pool_n, 3, ny, nx), dtype=torch.float64, device="cuda")
    ph = torch.empty_like(om)
    gen = [0]

    def exact_runs():
        gen[0] += 1
        return P.EpdLb([W.with_(r, seed=r.seed + 7777 * gen[0]) for r in runs])

    t0 = time.perf_counter()
    he, slot, age = exact_runs(), 0, 0
    while slot < pool_n:  # fill the pool
        he.step(1)
        age += 1
        for r in range(n_runs):
            if slot < pool_n:
                he.fields_dev(r, om[slot], ph[slot])
                slot += 1
    he.sync()
    s_in, s_out = S.scales_from(om[:64].cpu().numpy(), ph[:64].cpu().numpy())
    sm = S.Surrogate(runs[0], batch, s_in=s_in, s_out=s_out, seed=5)
    iters = max(1, pairs // n_runs)
    streamed = pool_n
    for it in range(iters):
        if age >= reseed:
            he.close()
            he, age = exact_runs(), 0
        he.step(1)
        age += 1
        # the pool slots written next may be the ones the last batch was
        # gathered from: the handle's stream waits for that gather
        he.stream.wait_stream(torch.cuda.current_stream())
        for r in range(n_runs):
            he.fields_dev(r, om[slot % pool_n], ph[slot % pool_n])
            slot += 1
        streamed += n_runs
        with torch.cuda.stream(he.stream):
            idx = torch.randint(0, pool_n, (batch,), device="cuda")
        torch.cuda.current_stream().wait_stream(he.stream)
        lr = 2e-3 * 0.5 * (1.0 + math.cos(math.pi * it / iters))
        loss = sm.train_step(om[idx], ph[idx], lr=lr)
    torch.cuda.synchronize()
    he.close()
    info = {"pairs_streamed": streamed, "pool": pool_n, "iterations": iters, "batch": batch,
            "reseed_every_steps": reseed, "seconds": time.perf_counter() - t0, "final_loss": float(loss.item()),
            "grid": f"{ny}x{nx}",
            "network": "4 layers, 32 channels, 3x3 kernels of dilation 1, 2, 2, 4, BF16 tensor-core "
                       "operands, FP32 accumulation; Phi(t+dt) from the tangent pass"}
    return sm, s_in, s_out, info


def evaluate_surrogate(P, torch, runs, sm, s_in, s_out, flush, timed_steps, eval_steps, exact_ms):
    """The stepper with the surrogate standing in (exact every 8th step,
    fallback above a relative residual of 0.2, the last exact force held on
    surrogate steps) timed over timed_steps, and its densities and velocity
    compared with an exact run from the same initial state after eval_steps
    steps, holding the force and, for comparison, with the surrogate's own."""
    import numpy as np

    tol = 0.2
    hb = P.EpdLb(runs)
    hb.set_surrogate(sm.params, s_in, s_out, exact_every=8, residual_tol=tol, hold_force=True)
    per, _ = time_steps(hb, hb.stream, timed_steps, flush)
    hb.sync()
    hb.close()
    ha = P.EpdLb(runs)
    ha.step(eval_steps)
    ha.sync()
    acc = {}
    for hold in (True, False):
        hc = P.EpdLb(runs)
        hc.set_surrogate(sm.params, s_in, s_out, exact_every=8, residual_tol=tol, hold_force=hold)
        hc.step(eval_steps)
        hc.sync()
        derr, drms, verr, vrms = [], [], [], []
        for r in range(len(runs)):
            pa, _ = ha.densities(r)
            pc, _ = hc.densities(r)
            for c in range(2):
                fl = pa[c] - pa[c].mean()
                derr.append(float(np.abs(pc[c] - pa[c]).max() / np.abs(fl).max()))
                drms.append(float(np.sqrt(((pc[c] - pa[c]) ** 2).mean() / (fl ** 2).mean())))
            va, vc = ha.velocity(r), hc.velocity(r)
            if np.abs(va).max() > 0:
                verr.append(float(np.abs(vc - va).max() / np.abs(va).max()))
                vrms.append(float(np.sqrt(((vc - va) ** 2).mean() / (va ** 2).mean())))
        acc[hold] = (derr, drms, verr, vrms, hc.surrogate_stats())
        hc.close()
    ha.close()
    derr, drms, verr, vrms, st = acc[True]
    ms = sum(per) / len(per)
    return {"ms_per_step": ms, "median_ms_per_step": float(np.median(per)), "steps": timed_steps,
            "exact_every": 8, "residual_tol": tol,
            "residual_definition": "RMS of Phi_sur - Phi_exact over the A and B densities at omega~, relative to the RMS "
                                   "fluctuation of the exact densities, max over runs, at every exact step",
            "value_equivalent": units_per_step(runs) / (ms * 1e-3),
            "speedup_vs_exact_mixed": exact_ms / ms,
            "density_error_vs_exact": max(derr), "density_rms_error_vs_exact": max(drms),
            "velocity_error_vs_exact": max(verr) if verr else None,
            "velocity_rms_error_vs_exact": max(vrms) if vrms else None, "eval_steps": eval_steps,
            "velocity_error_per_run": verr, "force": "held from the last exact step on surrogate steps",
            "with_surrogate_force": {"density_error_vs_exact": max(acc[False][0]),
                                     "velocity_error_vs_exact": max(acc[False][2]) if acc[False][2] else None,
                                     "velocity_error_per_run": acc[False][2]},
            "eval_stats": st,
            "density_error_definition": "max |Phi_sur - Phi_exact| / max |Phi_exact - <Phi_exact>| over runs and the A, B "
                                        "species after eval_steps steps, both runs from the same initial state (velocity: "
                                        "the same with u, relative to max |u|)"}


def bf16_peak():
    """(burst dense BF16 TFLOP/s, "measured" or "fallback")."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    except Exception:
        return 1900.0, "fallback"


def surrogate_rates(torch, sm, runs, flush, reps=10):
    """The surrogate's network kernels on the workload batch: CUDA-event time
    of one inference (the four tcgen05 convolutions and their small
    companions) and of one forward + tangent pass, L2 flushed before each;
    the convolutions' algorithmic BF16 FLOPs against the tensor-core peak."""
    import numpy as np

    nb, ny, nx = len(runs), runs[0].ny, runs[0].nx
    om = torch.from_numpy(1e-3 * np.random.default_rng(3).standard_normal((nb, 3, ny, nx))).cuda()
    om2 = om + 1e-6
    for _ in range(3):
        sm.tangent(om, om2)
    torch.cuda.synchronize()

    def timed(fn):
        ts = []
        for _ in range(reps):
            flush.add_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return float(np.median(ts))

    fwd = timed(lambda: sm.forward(om))
    tan = timed(lambda: sm.tangent(om, om2))
    # 2 x 9 taps x C_in x C_out per site and layer (the stored channel
    # counts the network computes: 3, 32, 32, 32 in; 32, 32, 32, 2 out)
    flops = 2.0 * nb * ny * nx * 9 * (3 * 32 + 32 * 32 + 32 * 32 + 32 * 2)
    peak, kind = bf16_peak()
    tf = flops / (fwd * 1e-3) / 1e12
    return {"batch": f"{nb} x {ny}x{nx}", "forward_ms": fwd, "forward_plus_tangent_ms": tan,
            "forward_tflops_algorithmic": tf, "bf16_peak_tflops": peak, "peak_kind": kind,
            "frac_of_bf16_peak": tf / peak}


def surrogate_section(P, W, torch, runs, flush, args, exact_ms):
    """The surrogate on the workload: trained on the workload's own runs
    (args.surrogate_pairs streamed pairs), evaluated on them."""
    sm, s_in, s_out, info = train_surrogate(P, W, torch, runs, args.surrogate_pairs)
    out = evaluate_surrogate(P, torch, runs, sm, s_in, s_out, flush, args.surrogate_steps, args.surrogate_eval_steps,
                             exact_ms)
    out["training"] = info
    out["network_kernels"] = surrogate_rates(torch, sm, runs, flush)
    return out


def group_concurrency(P, runs, flush, steps=10):
    """How much the step graph's per-group streams overlap: the median step
    of all runs in one handle (one graph, a stream per group) against the
    sum of the medians of every group stepped alone (L2 flushed before each
    timed step)."""
    import collections

    import numpy as np

    def median_step(rs):
        h = P.EpdLb(rs)
        h.step(2)
        h.sync()
        per, _ = time_steps(h, h.stream, steps, flush)
        h.close()
        return float(np.median(per))

    groups = collections.OrderedDict()
    for r in runs:
        groups.setdefault((r.ny, r.nx, r.ns), []).append(r)
    alone = {f"{ny}x{nx} N_s={ns}": median_step(rs) for (ny, nx, ns), rs in groups.items()}
    together = median_step(runs)
    return {"graph_ms": together, "groups": len(groups), "sum_of_groups_alone_ms": sum(alone.values()),
            "overlap": sum(alone.values()) / together, "groups_alone_ms": alone}


def config_section(P, W, torch, name, flush, args, rank):
    """Another configuration of the benchmark set, measured as the headline
    line: CUDA-event ms per step over args.config_steps steps (L2 flushed
    before each), the rates, the FP64-plain path over 2 steps and the MIXED
    path's error against it after them; the vesicle configuration also runs
    the surrogate, trained on 256 x 512 grids with its parameters (the
    network is a local operator of +-9 sites, so it carries over to the
    large grid) and evaluated on the 1024 x 2048 run."""
    import numpy as np

    runs = workload_runs(name, P.MIXED_FP32, rank)
    h = P.EpdLb(runs)
    h.step(2)
    h.sync()
    per, _ = time_steps(h, h.stream, args.config_steps, flush)
    h.close()
    ms = sum(per) / len(per)
    out = {"workload": WORKLOADS[name], "ms_per_step": ms, "value": units_per_step(runs) / (ms * 1e-3), "unit": UNIT,
           "lb_mlups": sites_per_step(runs) / (ms * 1e-3) / 1e6, "steps": args.config_steps}
    runs64 = workload_runs(name, P.PLAIN_FP64, rank)
    h64 = P.EpdLb(runs64)
    h64.step(1)
    h64.sync()
    per64, _ = time_steps(h64, h64.stream, 2, flush)
    ms64 = sum(per64) / len(per64)
    out["fp64_plain"] = {"ms_per_step": ms64, "value": units_per_step(runs64) / (ms64 * 1e-3), "steps": 2}
    out["speedup_vs_fp64_plain"] = ms64 / ms
    hm = P.EpdLb(runs)
    hm.step(3)
    out["mixed_error"] = precision_errors(hm, h64, len(runs), np)
    out["mixed_error"]["steps"] = 3
    hm.close()
    h64.close()
    if name == "ensemble32":
        out["concurrency"] = group_concurrency(P, runs, flush)
    if name == "vesicle" and args.surrogate_pairs > 0:
        train_runs = [W.with_(runs[0], nx=512, ny=256, seed=runs[0].seed + 31 * k) for k in range(4)]
        sm, s_in, s_out, info = train_surrogate(P, W, torch, train_runs, args.config_surrogate_pairs)
        # timed over whole cycles of the exact-every-8 schedule
        sur = evaluate_surrogate(P, torch, runs, sm, s_in, s_out, flush, 8 * max(2, -(-args.config_steps // 8)),
                                 args.config_eval_steps, ms)
        sur["training"] = info
        out["surrogate"] = sur
    return out


def exact_section(P, runs, flush, args):
    """The exact step of App. C (convection of Phi, Fletcher-Reeves inversion
    to the paper's 1e-8 tolerance) on the same workload: time per step and the
    iterations each run needed."""
    h = P.EpdLb(runs)
    h.step(args.warmup)
    h.set_inversion(100, 1e-8)
    h.step(1)
    h.sync()
    per, _ = time_steps(h, h.stream, args.exact_steps, flush)
    h.sync()
    stats = [h.inversion_stats(r) for r in range(len(runs))]
    h.close()
    return {"ms_per_step": float(sum(per) / len(per)), "steps": args.exact_steps, "tol": 1e-8, "max_iter": 100,
            "iterations_last_step": [s["iterations"] for s in stats],
            "residual0_last_step": [s["residual0"] for s in stats],
            "residual_last_step": [s["residual"] for s in stats],
            "note": "eager enqueue with one host synchronisation per CG iteration; per iteration two "
                    "single-chain solves (differential against the solve at the starting guess)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--surrogate-steps", type=int, default=40)
    ap.add_argument("--surrogate-pairs", type=int, default=50000,
                    help="exact (omega, Phi) pairs streamed through the surrogate's training (0 skips the surrogate)")
    ap.add_argument("--surrogate-eval-steps", type=int, default=1000,
                    help="steps after which the surrogate-driven run is compared with the exact run")
    ap.add_argument("--configs", default="ensemble32,vesicle",
                    help="other configurations measured into the line's configs key (comma list; empty: none)")
    ap.add_argument("--config-steps", type=int, default=5)
    ap.add_argument("--config-surrogate-pairs", type=int, default=64000)
    ap.add_argument("--config-eval-steps", type=int, default=200)
    ap.add_argument("--exact-steps", type=int, default=5,
                    help="steps of the exact step (CG inversion) timed on the same workload; 0 skips it")
    ap.add_argument("--workload", default="channel", choices=sorted(WORKLOADS),
                    help="channel (default): the 4 x 256x512 batch the metric is quoted on; ensemble32, "
                         "vesicle and paper150 (the paper's own 150x150 ensembles) are the other configurations")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return

    import numpy as np
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")

    import paper_1804_02883_gb300 as P
    from paper_1804_02883_gb300 import workloads as W

    P.lib()
    runs = workload_runs(args.workload, P.MIXED_FP32, rank)
    h = P.EpdLb(runs)
    h.enable_timing(True)
    stream = h.stream
    flush = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > 129 MB L2

    for _ in range(args.warmup):
        h.step(1)
    h.sync()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    barrier()
    with Clocks(local) as clk:
        t0 = time.perf_counter()
        per_step, kern = time_steps(h, stream, args.steps, flush, with_kernels=True)
        barrier()
        wall = time.perf_counter() - t0
    h.sync()
    dev_ms = max_over_ranks(float(sum(per_step)), dist, "cuda")
    value = job_rate(units_per_step(runs), args.steps, world, dev_ms * 1e-3)
    ms_per_step = dev_ms / args.steps
    lb_mlups = job_rate(sites_per_step(runs), args.steps, world, dev_ms * 1e-3) / 1e6

    # kernel durations inside the timed steps (event nodes in the step graph)
    nsite = sites_per_step(runs)
    tiles_path = h.tiles(0)["path"]
    n_launches = launches_per_step(runs, h)
    kt = {k: statistics.mean(d[k] for d in kern) for k in kern[0]}
    hbm, peak_kind = peaks()
    kernels = {}
    lb_bps = 88.0
    kernels["lb_collide_stream"] = {"ms": kt["lb_collide_stream"], "bytes_per_site": lb_bps,
                                    "achieved_gbs": lb_bps * nsite / (kt["lb_collide_stream"] * 1e-3) / 1e9}
    kernels["lb_collide_stream"]["frac"] = kernels["lb_collide_stream"]["achieved_gbs"] / hbm
    if "prop_cluster" in kt:
        # one cluster-resident launch = one single-chain solve of every run:
        # per run and contour step, forward + inverse transforms along both
        # axes, 10 n log2(n) flops (5 N log2 N per transform of length N)
        flops = sum(10.0 * r.nx * r.ny * math.log2(r.nx * r.ny) * r.ns for r in runs)
        tf = flops / (kt["prop_cluster"] * 1e-3) / 1e12
        peak_tf = FP32_SMS * FP32_LANES * 2 * FP32_MHZ * 1e6 / 1e12
        kernels["prop_cluster"] = {"ms": kt["prop_cluster"], "flops": flops, "achieved_tflops": tf, "frac": tf / peak_tf}
        # DRAM bytes (read + write) of the differential solve's chain launches
        # on this workload, from one ncu capture of the current kernels
        # (profiles/cluster_solve_channel_4x256x512_mixed.md): 8 phased
        # launches of 4 x 256 x 512, N_s = 64
        launches = h.tiles(0)["chain_launches"]
        traffic = CHAIN_DIFF_TRAFFIC_BYTES if (args.workload == "channel" and launches == 8) else None
        roofline = {"bound": "alu", "kernel": f"prop_chain (the step's second, differential single-chain solve of all "
                                              f"runs; {launches} launch(es) timed together)", "achieved": tf,
                    "peak": peak_tf, "unit": "TFLOP/s", "frac": tf / peak_tf, "traffic": traffic,
                    "peak_source": "derived FP32 peak: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz"}
    else:
        # streaming passes, per site and contour step (FP32 complex z = g + i g'):
        # radix-8 row pass = chain read 8 + write 8, factors 8, history store 8;
        # radix-2 row pass accumulating the contour sums also reads the history
        # and read-modify-writes the FP64 sums; column pass = chain read + write
        # MIXED (differential second solve, whose passes are the timed ones):
        # chain read + write 16, factors 8, rho 8, reference node 8, change
        # store 8 in every row pass
        radix8 = tiles_path == 1
        if h.tiles(0)["differential"]:
            bytes_per_site = {"prop_row_accumulate": 48.0, "prop_row_store": 48.0, "prop_col": 16.0}
        else:
            bytes_per_site = {"prop_row_accumulate": 32.0 if radix8 else 64.0, "prop_row_store": 32.0, "prop_col": 16.0}
        for k, bps in bytes_per_site.items():
            gbs = bps * nsite / (kt[k] * 1e-3) / 1e9
            kernels[k] = {"ms": kt[k], "bytes_per_site": bps, "achieved_gbs": gbs, "frac": gbs / hbm}
        dom = "prop_row_accumulate"
        name = ("prop_row8 (row pass of one contour step, radix-8 streaming" if radix8 else "prop_row (row pass, streaming") + \
            (", differential second solve)" if h.tiles(0)["differential"] else ")")
        roofline = {"bound": "hbm", "kernel": name, "achieved": kernels[dom]["achieved_gbs"], "peak": hbm,
                    "unit": "GB/s", "frac": kernels[dom]["achieved_gbs"] / hbm, "traffic": None,
                    "peak_source": f"{peak_kind} hbm_gbs (copy)"}

    # end to end through the C ABI with host buffers: upload omega of every
    # run from pinned memory, one step, read Phi and Q of every run back
    # (the asynchronous host-buffer calls, one synchronisation per step)
    host_om = [torch.empty(3 * r.nx * r.ny, dtype=torch.float64, pin_memory=True) for r in runs]
    host_phi = [torch.empty(3 * r.nx * r.ny, dtype=torch.float64, pin_memory=True) for r in runs]
    host_q = [torch.empty(2, dtype=torch.float64, pin_memory=True) for _ in runs]
    for k in range(len(runs)):
        om, _, _ = h.get_state(k)
        host_om[k].copy_(torch.from_numpy(om.ravel()))
    h.enable_timing(False)
    h.step(1)
    h.sync()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        for k in range(len(runs)):
            h.set_omega_async(k, host_om[k].data_ptr())
        h.step(1)
        for k in range(len(runs)):
            h.densities_async(k, host_phi[k].data_ptr(), host_q[k].data_ptr())
        h.sync()
    barrier()
    e2e_t = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    e2e = {"value": job_rate(units_per_step(runs), args.e2e_steps, world, e2e_t), "unit": UNIT,
           "h2d_bytes_per_step": int(sum(3 * r.nx * r.ny * 8 for r in runs)),
           "d2h_bytes_per_step": int(sum(3 * r.nx * r.ny * 8 + 16 for r in runs))}

    analysis = analysis_section(torch, h, runs, flush, hbm)
    cufft = None
    if "prop_cluster" in kt:
        try:
            cufft = cufft_section(torch, runs, h, kt["prop_cluster"], flush)
        except Exception as ex:  # a library comparison never costs the line
            cufft = {"unavailable": f"{type(ex).__name__}: {ex}"[:200]}

    # learned surrogate (exact every 8th step) on the same workload
    sur = None
    if args.surrogate_steps > 0 and args.surrogate_pairs > 0 and all(r.nx % 16 == 0 and r.ny % 16 == 0 for r in runs) and len({(r.nx, r.ny) for r in runs}) == 1:
        sur = surrogate_section(P, W, torch, runs, flush, args, ms_per_step)
    # FP64-plain path on the same workload
    h.close()
    del h
    exact = None
    if args.exact_steps > 0:
        try:
            exact = exact_section(P, runs, flush, args)
        except P.EpdLbError as e:  # grids without an exact MIXED path
            exact = {"unavailable": str(e)}
    fp64 = None
    if args.fp64_steps > 0:
        runs64 = workload_runs(args.workload, P.PLAIN_FP64, rank)
        h64 = P.EpdLb(runs64)
        h64.step(1)
        h64.sync()
        per64, _ = time_steps(h64, h64.stream, args.fp64_steps, flush)
        ms64 = sum(per64) / len(per64)
        fp64 = {"value": units_per_step(runs64) / (ms64 * 1e-3), "unit": UNIT, "ms_per_step": ms64,
                "lb_mlups": sites_per_step(runs64) / (ms64 * 1e-3) / 1e6, "steps": args.fp64_steps}
        # the MIXED path's error: a fresh MIXED batch stepped as often from the
        # same initial state as the FP64 one
        try:
            hm = P.EpdLb(runs)
            hm.step(1 + args.fp64_steps)
            fp64["mixed_error"] = precision_errors(hm, h64, len(runs), np)
            fp64["mixed_error"]["steps"] = 1 + args.fp64_steps
            hm.close()
        except Exception as ex:  # never costs the line
            fp64["mixed_error"] = {"unavailable": f"{type(ex).__name__}: {ex}"[:200]}
        h64.close()

    if sur is not None:
        sur["speedup_vs_fp64_plain"] = fp64["ms_per_step"] / sur["ms_per_step"] if fp64 else None
    configs = {}
    for name in [c for c in args.configs.split(",") if c and c != args.workload]:
        try:
            configs[name] = config_section(P, W, torch, name, flush, args, rank)
        except Exception as ex:  # a side configuration never costs the line
            configs[name] = {"unavailable": f"{type(ex).__name__}: {ex}"[:200]}
    line = None
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            import oracle as O

            O.build()
            rs = runs[min(1, len(runs) - 1)]
            t1 = oracle_step_time(rs, 1)
            cpu = {"value": rs.nx * rs.ny * rs.ns * 4 / t1, "unit": UNIT, "cores": 1,
                   "kind": "oracle", "sample": f"1 oracle coupled step of one {rs.ny}x{rs.nx} N_s={rs.ns} run",
                   "seconds": t1}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload],
                       "precision": "mixed (FP32 propagator, LB and EPD transforms; FP64 fields, contour sums, Q)",
                       "l2": "flushed (256 MB write) before every timed step", "parallelism": f"replicas x{world}"},
            "lb_mlups": lb_mlups,
            "fp64_plain": fp64,
            "speedup_vs_fp64_plain": value / fp64["value"] if fp64 else None,
            "wall_s": wall,
            "kernels": kernels,
            "roofline": roofline,
            "surrogate": sur,
            "configs": configs,
            "exact_step": exact,
            "analysis": analysis,
            "cufft_comparison": cufft,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": n_launches * args.steps,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
