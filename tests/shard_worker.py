"""One rank of the two-rank gloo test of sharding: trace this rank's
contiguous range of one run (single key, E_eff of the whole run) with the
oracle standing in for the GPU tracer, pool the tallies and statistics over
the ranks with the library's shard module, and write what this rank sees."""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import torch  # noqa: E402
import torch.distributed as dist  # noqa: E402

import oracle  # noqa: E402
from inputs import workloads as W  # noqa: E402
from paper_2104_03573_gb300 import _lib as L, shard  # noqa: E402


def stats_row(r):
    """The library's per-geometry stats layout, filled from an oracle result."""
    sc = r["scal"]
    row = np.zeros(L.NSTATS)
    row[L.STAT_KAPPA] = r["kappa"]
    row[L.STAT_Q_MEAN] = r["q_mean"]
    row[L.STAT_SUMX] = sc[oracle.SUMX]
    row[L.STAT_SUMX2] = sc[oracle.SUMX2]
    row[L.STAT_EVENTS] = sc[oracle.EVENTS]
    row[L.STAT_TRUNCATED] = sc[oracle.TRUNC]
    row[L.STAT_E_TOT] = sc[oracle.ETOT]
    row[L.STAT_MAX_EVENTS] = sc[oracle.MAXEV]
    row[L.STAT_KAPPA_CELL] = r["kappa_cell"]
    row[L.STAT_SIGNED_EMITTED] = sc[oracle.SIGNED_EMIT]
    row[L.STAT_SIGNED_ABSORBED] = sc[oracle.SIGNED_ABS]
    row[L.STAT_N] = r["n_traced"]
    row[L.STAT_ABSORBED] = sc[oracle.ABSORBED]
    return row


def main():
    rank, world, port, out_dir, n = (int(sys.argv[1]), int(sys.argv[2]), int(sys.argv[3]), sys.argv[4],
                                     int(sys.argv[5]))
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    wl = W.si_slab_c2(n=n, material=W.bvk_holland(n_per_branch=20))
    run = wl.run
    a, c = shard.shard_range(n, rank, world)
    r = oracle.run_steady(wl.material, wl.geometries[0], run, pid_begin=a, pid_end=a + c, n_total=n,
                          per_particle=True, n_threads=2)
    tallies = [torch.tensor(r["T"]), torch.tensor(r["q"]), torch.tensor(r["q_bin"])]
    shard.allreduce_tallies(tallies)
    pooled = shard.allreduce_stats(stats_row(r)[None, :])[0]
    t_max = shard.max_over_ranks(1.0 + rank)
    np.save(os.path.join(out_dir, f"pp{rank}.npy"), np.stack([r["events_pp"].astype(np.float64), r["X_pp"]]))
    if rank == 0:
        np.save(os.path.join(out_dir, "tallies.npy"),
                np.concatenate([t.numpy().ravel() for t in tallies]))
        with open(os.path.join(out_dir, "rank0.json"), "w") as f:
            json.dump({"stats": pooled.tolist(), "t_max": t_max}, f)
    dist.destroy_process_group()


if __name__ == "__main__":
    main()
