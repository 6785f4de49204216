"""Shared helpers of the GPU tests: run a workload through the C ABI and
return numpy results comparable with the oracle's."""
import math

import numpy as np

from inputs import workloads as W


def steady_cfg(api, L, run, precision, seed=None, **kw):
    return api.SteadyConfig(seed=run.seed if seed is None else seed, precision=precision,
                            n_scat_max=run.n_scat_max, max_events=kw.pop("max_events", run.max_events),
                            n_cells=run.n_cells, cell_axis=run.cell_axis, tally_axis=run.tally_axis,
                            per_bin=run.per_bin, **kw)


def gpu_steady(mat, geoms, ns, run, precision, seed=None, per_particle=False, M=None, **kw):
    import torch
    from paper_2104_03573_gb300 import api, _lib as L
    M = M or api.Material(mat)
    Gs = [api.Geometry(g) for g in geoms]
    cfg = steady_cfg(api, L, run, precision, seed, **kw)
    out = api.run_steady(M, Gs, ns, cfg, per_particle=per_particle)
    torch.cuda.synchronize()
    r = {"stats": out.stats.cpu().numpy()}
    if out.T is not None:
        r["T"] = out.T.cpu().numpy()
        r["q"] = out.q.cpu().numpy()
    if out.q_bin is not None:
        r["q_bin"] = out.q_bin.cpu().numpy()
    if per_particle:
        r["events_pp"] = out.events_pp.cpu().numpy().astype(np.uint32)
        r["X_pp"] = out.X_pp.cpu().numpy()
    return r


def gpu_transient(mat, geom, run, precision, seed=None, per_particle=False, **kw):
    import torch
    from paper_2104_03573_gb300 import api
    M = api.Material(mat)
    G = api.Geometry(geom)
    cfg = api.TransientConfig(seed=run.seed if seed is None else seed, t_max=run.t_max, t_meas=run.t_meas,
                              grid=run.grid, precision=precision, max_events=run.max_events,
                              regions=getattr(run, "regions", ()),
                              time_average=bool(getattr(run, "time_average", False)), **kw)
    out = api.run_transient(M, G, run.n, cfg, per_particle=per_particle)
    torch.cuda.synchronize()
    r = {"tally": out.tally.cpu().numpy(), "stats": out.stats.cpu().numpy()}
    if per_particle:
        r["events_pp"] = out.events_pp.cpu().numpy().astype(np.uint32)
    return r


def rel_close(a, b, rtol):
    """max |a - b| <= rtol * max |b| (vector-wide relative error)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    scale = max(np.max(np.abs(b)), 1e-300)
    err = np.max(np.abs(a - b)) if a.size else 0.0
    return err <= rtol * scale, err / scale


def z_scores(m1, s1, m2, s2):
    s = np.sqrt(np.asarray(s1) ** 2 + np.asarray(s2) ** 2)
    ok = s > 0
    z = np.zeros_like(np.asarray(m1, dtype=np.float64))
    z[ok] = (np.asarray(m1)[ok] - np.asarray(m2)[ok]) / s[ok]
    return z


def batch_stats(vals):
    v = np.asarray(vals)
    return v.mean(axis=0), v.std(axis=0, ddof=1) / math.sqrt(v.shape[0])
