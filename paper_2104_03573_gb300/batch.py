"""Batched multi-geometry steady runs under a captured CUDA graph.

All geometries of a batch (for example dozens of film thicknesses with
uneven particle counts) are traced by one persistent launch: the flattened
particle index space is shared by every lane of the GPU through one work
counter, so uneven per-geometry work balances itself.  The whole run
(scratch clear, setup kernel, tracing kernel, finalisation) is captured once
into a CUDA graph and replayed; the Philox key lives in a device tensor, so
every replay after a key update traces an independent sample.
"""
from __future__ import annotations

from dataclasses import replace
from typing import Optional, Sequence

import numpy as np

from . import _lib as L
from . import api, autotune


class GraphBatch:
    def __init__(self, material: api.Material, geoms: Sequence[api.Geometry], n_particles,
                 cfg: api.SteadyConfig, tune: bool = True):
        import torch
        self.material = material
        self.geoms = list(geoms)
        self.n = np.ascontiguousarray(np.asarray(n_particles, dtype=np.uint64))
        if tune and cfg.precision == L.FP32_TRACE:
            cfg = replace(autotune.tune(material, self.geoms, self.n, replace(cfg, trace_events=None)),
                          trace_events=cfg.trace_events)
        self.seed = torch.tensor([int(cfg.seed)], dtype=torch.int64, device="cuda")
        # trace events, if given, become event-record nodes of the graph
        self.cfg = replace(cfg, seed_device=self.seed)
        ws = api.steady_workspace_size(material, self.geoms, self.n, self.cfg)
        self.workspace = torch.empty(ws, dtype=torch.uint8, device="cuda")
        self.out = api.SteadyOutputs(len(self.geoms), material.n_bins, cfg.n_cells, cfg.per_bin, regions=cfg.regions,
                                     nscat=cfg.n_scat_max if cfg.nscat_curve else 0, det_per_bin=cfg.det_per_bin)
        self.stream = torch.cuda.Stream()
        self.stream.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(self.stream):
            self._run()                      # first run outside capture (lazy module / attribute set-up)
        torch.cuda.current_stream().wait_stream(self.stream)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=self.stream, capture_error_mode="thread_local"):
            self._run()

    def _run(self):
        api.run_steady(self.material, self.geoms, self.n, self.cfg, out=self.out, workspace=self.workspace)

    def replay(self, seed: Optional[int] = None) -> api.SteadyOutputs:
        """Run the captured batch once (asynchronously on the current stream)
        with Philox key `seed` (default: previous key + 1)."""
        if seed is None:
            self.seed.add_(1)
        else:
            self.seed.fill_(int(seed))
        self.graph.replay()
        return self.out
