"""One rank of the replica (N > 1) path of bench.py on CPU with gloo: launched
by tests/test_replicas.py through torch.distributed.run, two ranks.  Checks
the max-over-ranks timing, the whole-job rate and that every rank steps
its own, differently seeded batch."""
import os
import sys

import torch.distributed as dist

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import paper_1804_02883_gb300 as P  # noqa: E402


def main() -> None:
    dist.init_process_group("gloo")
    rank, world = dist.get_rank(), dist.get_world_size()
    assert world == 2
    # the slowest rank sets the time
    t = bench.max_over_ranks(10.0 + 5.0 * rank, dist)
    assert t == 15.0, t
    # whole-job rate: both ranks' units over the slowest rank's time
    assert bench.job_rate(100.0, 4, world, 2.0) == 400.0
    # replicas: the same configuration on every rank, different seeds
    for name in ("channel", "ensemble32", "paper150"):
        runs = bench.workload_runs(name, P.MIXED_FP32, rank)
        mine = [r.seed for r in runs]
        shapes = [(r.nx, r.ny, r.ns, r.f0) for r in runs]
        gathered = [None] * world
        dist.all_gather_object(gathered, (mine, shapes))
        (s0, sh0), (s1, sh1) = gathered
        assert sh0 == sh1, name
        assert not set(s0) & set(s1), name
    dist.barrier()
    dist.destroy_process_group()
    print(f"rank {rank} ok", flush=True)


if __name__ == "__main__":
    main()
