"""Sharding of steady runs over ranks (one GPU per rank).

Particles are independent (the paper's parallelisation is over particles,
Sec. 6).  A run of N particles of a geometry is split into contiguous ranges
of particle indices, one per rank; every particle draws from Philox with its
own index under the run's one key (``pid_begin`` in the run parameters) and
every call scales its tallies by the whole run's E_eff = E_tot / N
(``n_total``).  The ranks therefore trace exactly the particles of the
single-GPU run, and the result does not depend on the partition.  Nothing is
exchanged on the data path; after the run one sum-reduction combines the
tallies (T, q, q_bin, detector sums) and the per-geometry statistics:
kappa, q_mean, sum X, sum X^2, the event and particle counts add up, the
largest event count and the worst status are kept, and the standard errors
follow from the pooled sum X, sum X^2 and N.  Timing is the maximum over
ranks.
"""
from __future__ import annotations

import math
from dataclasses import replace
from typing import Dict, List, Sequence, Tuple

import numpy as np

from . import _lib as L

# statistics that add up over the ranks of a split run
_ADD = (L.STAT_KAPPA, L.STAT_Q_MEAN, L.STAT_SUMX, L.STAT_SUMX2, L.STAT_EVENTS, L.STAT_TRUNCATED,
        L.STAT_KAPPA_CELL, L.STAT_SIGNED_EMITTED, L.STAT_SIGNED_ABSORBED, L.STAT_N, L.STAT_ABSORBED)


KEY_STRIDE = 1_000_003


def rank_key(seed: int, rank: int) -> int:
    """Philox key of `rank`'s independent sample, for runs that cannot be
    split by particle index (transient runs): rank r uses seed + 1000003 r."""
    return int(seed) + KEY_STRIDE * int(rank)


def shard_range(n_total: int, rank: int, world: int) -> Tuple[int, int]:
    """(first particle index, particle count) of `rank`'s contiguous range."""
    a = n_total * rank // world
    b = n_total * (rank + 1) // world
    return a, b - a


def rank_config(cfg, n_total: Sequence[int], rank: int, world: int):
    """`cfg` restricted to `rank`'s ranges of a run with n_total particles per
    geometry; returns (config, particles per geometry of this rank)."""
    ranges = [shard_range(int(n), rank, world) for n in n_total]
    cfg = replace(cfg, pid_begin=[a for a, _ in ranges], n_total=[int(n) for n in n_total])
    return cfg, [c for _, c in ranges]


def _status(codes) -> float:
    codes = set(float(c) for c in codes)
    for c in (L.ERR_REPLAY, L.ERR_TIMEOUT, L.WARN_TRUNCATED):
        if float(c) in codes:
            return float(c)
    return 0.0


def _finish(row: np.ndarray, q_per_x: float, k_per_q: float) -> np.ndarray:
    """Standard errors of a pooled stats row: q_se = (E_eff / V) sqrt(n var),
    with E_eff / V = q_mean / sum X (the same on every rank)."""
    n, sx, sx2 = row[L.STAT_N], row[L.STAT_SUMX], row[L.STAT_SUMX2]
    mean = sx / n if n else 0.0
    var = (sx2 - n * mean * mean) / (n - 1) if n > 1 else 0.0
    row[L.STAT_Q_SE] = abs(q_per_x) * math.sqrt(max(var, 0.0) * n)
    row[L.STAT_KAPPA_SE] = abs(k_per_q) * row[L.STAT_Q_SE]
    return row


def _ratios(rows: Sequence[np.ndarray]) -> Tuple[float, float]:
    q_per_x = next((r[L.STAT_Q_MEAN] / r[L.STAT_SUMX] for r in rows if r[L.STAT_SUMX] != 0.0), 0.0)
    k_per_q = next((r[L.STAT_KAPPA] / r[L.STAT_Q_MEAN] for r in rows if r[L.STAT_Q_MEAN] != 0.0), 0.0)
    return q_per_x, k_per_q


def combine_stats(rows: Sequence[np.ndarray]) -> np.ndarray:
    """Pool the stats rows (one geometry) of the calls that cover a run."""
    rows = [np.asarray(r, dtype=np.float64) for r in rows]
    out = rows[0].copy()
    for k in _ADD:
        out[k] = float(np.sum([r[k] for r in rows]))
    out[L.STAT_MAX_EVENTS] = max(r[L.STAT_MAX_EVENTS] for r in rows)
    out[L.STAT_STATUS] = _status(r[L.STAT_STATUS] for r in rows)
    return _finish(out, *_ratios(rows))


def _dev(group):
    import torch
    import torch.distributed as dist
    return torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" else "cpu"


def allreduce_stats(stats: np.ndarray, group=None) -> np.ndarray:
    """Pool [n_geoms][NSTATS] stats over the ranks of `group` (gloo: CPU
    tensors; nccl: the current device)."""
    import torch
    import torch.distributed as dist
    stats = np.atleast_2d(np.asarray(stats, dtype=np.float64))
    dev = _dev(group)
    world = dist.get_world_size(group)
    t = torch.tensor(stats, dtype=torch.float64, device=dev)
    gathered = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(gathered, t, group=group)
    per_rank = [g.cpu().numpy() for g in gathered]
    return np.stack([combine_stats([pr[g] for pr in per_rank]) for g in range(stats.shape[0])])


def allreduce_tallies(tensors: List, group=None) -> None:
    """Sum-reduce tally tensors in place (T, q, q_bin, detector sums) over
    the ranks of `group`; None entries are skipped."""
    import torch.distributed as dist
    for t in tensors:
        if t is None:
            continue
        if dist.get_backend(group) == "nccl" or t.device.type == "cpu":
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        else:                                  # gloo reduces host tensors
            h = t.cpu()
            dist.all_reduce(h, op=dist.ReduceOp.SUM, group=group)
            t.copy_(h)


def allreduce_steady(out, group=None) -> None:
    """Combine a rank's SteadyOutputs over the ranks of `group` in place: the
    tallies summed, the statistics pooled (see combine_stats)."""
    import torch
    allreduce_tallies([out.T, out.q, out.q_bin, getattr(out, "det", None)], group)
    pooled = allreduce_stats(out.stats.cpu().numpy(), group)
    out.stats.copy_(torch.as_tensor(pooled, dtype=out.stats.dtype, device=out.stats.device))


def pooled_kappa(stats_row: np.ndarray) -> Dict[str, float]:
    return {"kappa": float(stats_row[L.STAT_KAPPA]), "kappa_se": float(stats_row[L.STAT_KAPPA_SE]),
            "n": float(stats_row[L.STAT_N]), "events": float(stats_row[L.STAT_EVENTS])}


def max_over_ranks(x: float, group=None) -> float:
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=_dev(group))
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def sum_over_ranks(x: float, group=None) -> float:
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=_dev(group))
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return float(t.item())
