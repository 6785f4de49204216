"""One rank of the two-rank gloo test of independent-sample sharding: trace
this rank's sample with the oracle, pool the kappa accumulators and the
timings over the ranks, and write what rank 0 sees."""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import torch.distributed as dist  # noqa: E402

import oracle  # noqa: E402
from inputs import workloads as W  # noqa: E402
from paper_2104_03573_gb300 import _lib as L, shard  # noqa: E402


def stats_row(r, n):
    row = np.zeros(L.NSTATS)
    row[L.STAT_N] = n
    row[L.STAT_SUMX] = r["scal"][oracle.SUMX]
    row[L.STAT_SUMX2] = r["scal"][oracle.SUMX2]
    row[L.STAT_EVENTS] = r["events"]
    row[L.STAT_KAPPA] = r["kappa"]
    return row


def main():
    rank, world, port, out, n = int(sys.argv[1]), int(sys.argv[2]), int(sys.argv[3]), sys.argv[4], int(sys.argv[5])
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    wl = W.gray_slab_c1(n=n)
    run = wl.run
    run.seed = shard.rank_key(run.seed, rank)
    r = oracle.run_steady(wl.material, wl.geometries[0], run, n_threads=2)
    pooled = shard.allreduce_steady_stats(stats_row(r, n))
    t_max = shard.max_over_ranks(1.0 + rank)
    ev = shard.sum_over_ranks(r["events"])
    if rank == 0:
        with open(out, "w") as f:
            json.dump({"pooled": pooled, "t_max": t_max, "events": ev}, f)
    dist.destroy_process_group()


if __name__ == "__main__":
    main()
