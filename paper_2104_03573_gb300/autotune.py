"""Launch-shape autotuner of the persistent FP32 tracer.

For a given material / geometry batch / run configuration it times a
reduced-size run for each candidate (block size, blocks per SM, warp refill
threshold, and whether the run's last particles go to the tail kernel) and
keeps the fastest by particle-events per second.  Results are cached per
process by the features that decide the kernel variant and its load balance:
the material's and every geometry's content, the tallies, the extended
physics.  The physics does not depend on the choice: every particle's random
stream is keyed by its own id, so any launch shape produces the same
per-particle trajectories.
"""
from __future__ import annotations

from dataclasses import replace
from typing import Dict, Iterable, Optional, Sequence, Tuple

import numpy as np

from . import _lib as L
from . import api

_CACHE: Dict[tuple, dict] = {}

SHAPES: Tuple[Tuple[int, int, int], ...] = (
    (1024, 0, 4), (1024, 0, 8), (1024, 0, 1), (768, 0, 4), (768, 0, 1), (512, 0, 4), (256, 0, 1),
)
# (threads_per_block, blocks_per_sm, refill_threshold, tail_lanes): every
# shape without the tail kernel (-1) and with it (0, the default threshold)
DEFAULT_CANDIDATES: Tuple[Tuple[int, int, int, int], ...] = tuple(s + (t,) for s in SHAPES for t in (-1, 0))


def _key(material: api.Material, geoms: Sequence[api.Geometry], n_particles, cfg: api.SteadyConfig) -> tuple:
    n = np.asarray(n_particles, dtype=np.int64)
    return (getattr(material, "features", material.n_bins), tuple(getattr(g, "features", None) for g in geoms),
            int(cfg.n_cells), int(cfg.cell_axis), bool(cfg.cell_flux_axis), bool(cfg.per_bin), int(cfg.n_scat_max),
            int(cfg.tally_axis), bool(cfg.nscat_curve), len(cfg.regions or ()), bool(cfg.det_per_bin),
            int(cfg.tail_lanes), int(np.log2(max(1, int(n.sum())))))


def tune(material: api.Material, geoms: Sequence[api.Geometry], n_particles, cfg: api.SteadyConfig, *,
         fraction: float = 0.25, min_particles: int = 20_000, repeats: int = 2,
         candidates: Optional[Iterable[Tuple[int, ...]]] = None, verbose: bool = False) -> api.SteadyConfig:
    """Return `cfg` with the fastest (threads_per_block, blocks_per_sm,
    refill_threshold, tail_lanes) for this workload (FP32 path only); a
    tail_lanes the caller set (non-zero) is kept.  The sample must hold tens
    of particles per resident lane, or the drain tail of the persistent
    launch, not its steady state, decides the ranking."""
    import torch
    if cfg.precision != L.FP32_TRACE:
        return cfg
    key = _key(material, geoms, n_particles, cfg)
    if key in _CACHE:
        return replace(cfg, **_CACHE[key])
    n = np.asarray(n_particles, dtype=np.int64)
    sample = np.maximum(1, np.maximum((n * fraction).astype(np.int64), min(min_particles, int(n.max())) // len(n)))
    best, best_rate = None, -1.0
    results = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    cands = []
    for cand in (candidates or DEFAULT_CANDIDATES):
        cand = tuple(cand) + ((0,) if len(cand) == 3 else ())
        if cfg.tail_lanes != 0:
            cand = cand[:3] + (int(cfg.tail_lanes),)
        if cand not in cands:
            cands.append(cand)
    for threads, bps, refill, tail in cands:
        c = replace(cfg, threads_per_block=threads, blocks_per_sm=bps, refill_threshold=refill, tail_lanes=tail,
                    trace_events=None, seed_device=None)
        out = api.SteadyOutputs(len(geoms), material.n_bins, c.n_cells, c.per_bin, regions=c.regions,
                                nscat=c.n_scat_max if c.nscat_curve else 0, det_per_bin=c.det_per_bin)
        api.run_steady(material, geoms, sample, c, out=out)        # warm-up / first-launch costs
        times = []
        for _ in range(repeats):
            e0.record()
            api.run_steady(material, geoms, sample, c, out=out)
            e1.record()
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
        events = float(out.stats[:, L.STAT_EVENTS].sum().item())
        rate = events / min(times)
        results.append(((threads, bps, refill, tail), rate))
        if rate > best_rate:
            best, best_rate = (threads, bps, refill, tail), rate
    if verbose:
        for cand, rate in results:
            print(f"autotune {cand}: {rate:.3e} events/s")
    choice = {"threads_per_block": best[0], "blocks_per_sm": best[1], "refill_threshold": best[2],
              "tail_lanes": best[3]}
    _CACHE[key] = choice
    return replace(cfg, **choice)


def clear_cache() -> None:
    _CACHE.clear()
