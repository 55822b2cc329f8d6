"""Run a few coupled steps of a benchmark workload without timing or L2
flushes, for kernel profilers:

    python -m paper_1804_02883_gb300.profile_case --workload channel --steps 2

--exact N then runs N exact steps (Fletcher-Reeves inversion to the 1e-8
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
    "plain_small": lambda: [W.plain_small()],
    "paper150": lambda: W.paper_150(B.MIXED_FP32),
}


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="channel", choices=sorted(WORKLOADS))
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--exact", type=int, default=0, help="then this many exact steps (0: none)")
    args = ap.parse_args()
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
