"""Independent-sample sharding of steady runs over ranks (one GPU per rank).

Particles are independent (the paper's parallelisation is over particles,
Sec. 6), so N ranks each trace their own sample and nothing is exchanged on
the data path.  Each rank keys its Philox streams with its own key (rank r
uses seed + KEY_STRIDE * r), so no two ranks share a random word.  After the
run the ranks combine the per-particle accumulators of the estimator: the
kappa estimator is linear in sum_p X_p (Eq. flux_x_steady) with the common
constant c = kappa_r N_r / sum X_r of every rank, and its standard error
follows from the pooled sum X and sum X^2.  Timing is the maximum over ranks.
"""
from __future__ import annotations

import math
from typing import Dict, Sequence

import numpy as np

from . import _lib as L

KEY_STRIDE = 1_000_003


def rank_key(seed: int, rank: int) -> int:
    """Philox key of `rank`'s independent sample."""
    return int(seed) + KEY_STRIDE * int(rank)


def _pack(row: np.ndarray) -> np.ndarray:
    """[N, sum X, sum X^2, events, c] of one geometry's stats row."""
    n, sx = float(row[L.STAT_N]), float(row[L.STAT_SUMX])
    c = float(row[L.STAT_KAPPA]) * n / sx if sx != 0.0 else 0.0
    return np.array([n, sx, float(row[L.STAT_SUMX2]), float(row[L.STAT_EVENTS]), c])


def _finish(tot: np.ndarray, c: float) -> Dict[str, float]:
    n, sx, sx2, ev = (float(x) for x in tot[:4])
    mean = sx / n
    var = (sx2 - n * mean * mean) / (n - 1) if n > 1 else 0.0
    return {"n": n, "events": ev, "kappa": c * mean, "kappa_se": abs(c) * math.sqrt(max(var, 0.0) / n)}


def combine_steady_stats(rows: Sequence[np.ndarray]) -> Dict[str, float]:
    """Pool the stats rows (one geometry) of independent samples in one process."""
    packs = [_pack(np.asarray(r)) for r in rows]
    tot = np.sum([p[:4] for p in packs], axis=0)
    c = next((p[4] for p in packs if p[4] != 0.0), 0.0)
    return _finish(tot, c)


def allreduce_steady_stats(row: np.ndarray, group=None) -> Dict[str, float]:
    """Pool one geometry's stats row over the ranks of `group` (any backend;
    the reduction runs on a CPU tensor for gloo, on the current device for
    nccl)."""
    import torch
    import torch.distributed as dist
    p = _pack(np.asarray(row))
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor(p[:4], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return _finish(t.cpu().numpy(), p[4])


def max_over_ranks(x: float, group=None) -> float:
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def sum_over_ranks(x: float, group=None) -> float:
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return float(t.item())
