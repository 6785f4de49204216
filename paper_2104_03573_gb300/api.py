"""Python entry points of the MCBTE GB300 library (one per C-ABI call).

PyTorch supplies device memory and streams; the functions below only
marshal arguments into the C structures of ``include/mcbte.h`` and call the
CUDA library.  There is no CPU fallback: without the built library or a
CUDA device every call raises.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass
from typing import Dict, List, Optional, Sequence

import numpy as np

from . import _lib as L


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


class Material:
    """Device material tables built by ``mcbte_material_create``."""

    def __init__(self, m):
        lib = L.load()
        self._keep = [_f64(m.omega), _f64(m.v), _f64(m.tau)]
        d = L.MaterialDesc()
        d.n_bins = int(m.omega.shape[0])
        d.omega, d.v, d.tau = (a.ctypes.data for a in self._keep)
        if m.C is not None:
            c = _f64(m.C)
            self._keep.append(c)
            d.C = c.ctypes.data
        else:
            D, dw = _f64(m.D), _f64(m.domega)
            self._keep += [D, dw]
            d.D, d.domega = D.ctypes.data, dw.ctypes.data
        d.T_lin = float(m.T_lin)
        if getattr(m, "tau_imp", None) is not None:
            ti = _f64(m.tau_imp)
            self._keep.append(ti)
            d.tau_imp = ti.ctypes.data
        if getattr(m, "spec_bin", None) is not None:
            sb = _f64(m.spec_bin)
            self._keep.append(sb)
            d.spec_bin = sb.ctypes.data
        h = C.c_void_p()
        L.check(lib.mcbte_material_create(C.byref(d), C.byref(h)))
        self.handle = h
        self.n_bins = d.n_bins
        # what decides the tracer's kernel variant and load balance (the
        # autotuner's cache key): size, optional columns, the tables' content
        self.features = (d.n_bins, d.tau_imp is not None, d.spec_bin is not None,
                         hash(b"".join(a.tobytes() for a in self._keep)))
        self._keep = None

    def tables(self) -> Dict[str, np.ndarray]:
        n = self.n_bins
        Cb = np.zeros(n); prob = np.zeros(3 * n); thr = np.zeros(3 * n, dtype=np.uint64)
        al = np.zeros(3 * n, dtype=np.int32); sums = np.zeros(3)
        L.check(L.load().mcbte_material_tables(self.handle, Cb.ctypes.data, prob.ctypes.data, thr.ctypes.data,
                                               al.ctypes.data, sums.ctypes.data))
        return {"C": Cb, "prob": prob.reshape(3, n), "thr": thr.reshape(3, n), "alias": al.reshape(3, n),
                "C_tot": sums[0], "sum_Cv": sums[1], "sum_C_over_tau": sums[2]}

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and L._lib is not None:
            L._lib.mcbte_material_destroy(h)
            self.handle = None


def geometry_desc(g) -> "L.GeometryDesc":
    d = L.GeometryDesc()
    d.L[:] = [float(x) for x in g.L]
    d.face_type[:] = [int(x) for x in g.face_type]
    d.face_T[:] = [float(x) for x in g.face_T]
    d.face_p[:] = [float(x) for x in g.face_p]
    d.T_eq = float(g.T_eq)
    d.grad_T[:] = [float(x) for x in g.grad_T]
    d.pore = int(g.pore)
    d.pore_c[:] = [float(x) for x in g.pore_c]
    d.pore_r = float(g.pore_r)
    d.pore_p = float(g.pore_p)
    d.gauss = int(g.gauss)
    d.gauss_c[:] = [float(x) for x in g.gauss_c]
    d.gauss_sigma = float(g.gauss_sigma)
    d.gauss_dT = float(g.gauss_dT)
    inner = list(getattr(g, "inner", ()) or ())
    d.n_inner = len(inner)
    for k, seg in enumerate(inner[:16]):
        d.inner[k][:] = [float(c) for c in seg]
        d.inner_n[k][:] = [float(c) for c in g.inner_n[k]]
        d.inner_p[k] = float(g.inner_p[k])
    return d


class Geometry:
    """Geometry handle of ``mcbte_geometry_create``."""

    def __init__(self, g):
        d = geometry_desc(g)
        h = C.c_void_p()
        L.check(L.load().mcbte_geometry_create(C.byref(d), C.byref(h)))
        self.handle = h
        self.features = hash(bytes(d))   # the whole descriptor (autotuner cache key)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and L._lib is not None:
            L._lib.mcbte_geometry_destroy(h)
            self.handle = None


def _stream_ptr(stream) -> Optional[int]:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _ptr(t) -> Optional[int]:
    return None if t is None else t.data_ptr()


@dataclass
class SteadyConfig:
    seed: int
    precision: int = L.FP32_TRACE
    n_scat_max: int = 0
    max_events: int = 0
    n_cells: int = 0
    cell_axis: int = 2
    tally_axis: int = 2
    per_bin: bool = False
    threads_per_block: int = 0
    blocks_per_sm: int = 0
    time_budget_s: float = 0.0
    trace_events: Optional[tuple] = None     # (start, stop) torch.cuda.Event around the trace kernel
    seed_device: Optional[object] = None     # int64 device tensor holding the Philox key
    refill_threshold: int = 0
    cell_flux_axis: bool = False             # FP32 cell tallies: T and the tally-axis flux only
    regions: Sequence = ()                   # detector regions ((xmin..zmax) m, (nx, ny, nz)), one geometry
    nscat_curve: bool = False                # also kappa for every N_scat_max' <= n_scat_max (kappa_nscat)
    det_per_bin: bool = False                # detector outputs per frequency bin (det: [n_det][n_bins][4])
    tail_lanes: int = 0                      # FP32 tail: warps with <= this many particles left draw ahead (0: 8, -1: off)
    pid_begin: Sequence = ()                 # per geometry: index of this call's first particle in the run
    n_total: Sequence = ()                   # per geometry: particles of the whole run (E_eff normalisation)


def _event_handles(pair):
    if not pair:
        return None, None
    for e in pair:
        if not e.cuda_event:
            e.record()          # torch creates the CUDA event at its first record
    return pair[0].cuda_event, pair[1].cuda_event


def steady_params(cfg: SteadyConfig, n_particles: np.ndarray) -> "L.SteadyParams":
    p = L.SteadyParams()
    p.n_particles = n_particles.ctypes.data
    p.seed = int(cfg.seed)
    p.precision = int(cfg.precision)
    p.n_scat_max = int(cfg.n_scat_max)
    p.max_events = int(cfg.max_events)
    p.n_cells = int(cfg.n_cells)
    p.cell_axis = int(cfg.cell_axis)
    p.tally_axis = int(cfg.tally_axis)
    p.per_bin = int(bool(cfg.per_bin))
    p.threads_per_block = int(cfg.threads_per_block)
    p.blocks_per_sm = int(cfg.blocks_per_sm)
    p.time_budget_s = float(cfg.time_budget_s)
    p.trace_event_start, p.trace_event_stop = _event_handles(cfg.trace_events)
    p.seed_device = None if cfg.seed_device is None else cfg.seed_device.data_ptr()
    p.refill_threshold = int(cfg.refill_threshold)
    p.cell_flux_axis = int(bool(cfg.cell_flux_axis))
    p.nscat_curve = int(bool(cfg.nscat_curve))
    p.det_per_bin = int(bool(cfg.det_per_bin))
    p.tail_lanes = int(cfg.tail_lanes)
    keep = []
    if len(cfg.pid_begin):
        pb = np.ascontiguousarray(cfg.pid_begin, dtype=np.uint64)
        keep.append(pb)
        p.pid_begin = pb.ctypes.data
    if len(cfg.n_total):
        nt = np.ascontiguousarray(cfg.n_total, dtype=np.uint64)
        keep.append(nt)
        p.n_total = nt.ctypes.data
    p._keep_split = keep                    # host arrays read during the call
    regions = list(cfg.regions or ())
    if regions:
        boxes = np.ascontiguousarray([r[0] for r in regions], dtype=np.float64)
        grids = np.ascontiguousarray([r[1] for r in regions], dtype=np.int32)
        p._keep = (boxes, grids)            # host arrays read during the call
        p.n_regions, p.regions, p.region_grid = len(regions), boxes.ctypes.data, grids.ctypes.data
    return p


class SteadyOutputs:
    """Caller-owned device outputs of a steady run (torch tensors)."""

    def __init__(self, n_geoms: int, n_bins: int, n_cells: int, per_bin: bool, total: int = 0,
                 per_particle: bool = False, device=None, regions: Sequence = (), nscat: int = 0,
                 det_per_bin: bool = False):
        import torch
        dev = device or torch.device("cuda")
        f = dict(dtype=torch.float64, device=dev)
        nd = sum(int(np.prod(r[1])) for r in regions) if regions else 0
        # T, q_x, q_y, q_z per detector (and bin)
        self.det = (torch.zeros(nd, n_bins, 4, **f) if det_per_bin else torch.zeros(nd, 4, **f)) if nd else None
        self.T = torch.zeros(n_geoms, n_cells, **f) if n_cells > 0 else None
        self.q = torch.zeros(n_geoms, n_cells, 3, **f) if n_cells > 0 else None
        self.q_bin = torch.zeros(n_geoms, n_bins, **f) if per_bin else None
        self.stats = torch.zeros(n_geoms, L.NSTATS, **f)
        self.events_pp = torch.zeros(total, dtype=torch.int32, device=dev) if per_particle else None
        self.X_pp = torch.zeros(total, **f) if per_particle else None
        # kappa and its SE for N_scat_max = k + 1 at [g, k]
        self.kappa_nscat = torch.zeros(n_geoms, nscat, 2, **f) if nscat > 0 else None

    def struct(self) -> "L.SteadyOut":
        o = L.SteadyOut()
        o.T, o.q, o.q_bin, o.stats = _ptr(self.T), _ptr(self.q), _ptr(self.q_bin), _ptr(self.stats)
        o.events_pp, o.X_pp = _ptr(self.events_pp), _ptr(self.X_pp)
        o.det = _ptr(self.det)
        o.kappa_nscat = _ptr(self.kappa_nscat)
        o.on_host = 0
        return o


def _handles(objs) -> C.Array:
    arr = (C.c_void_p * len(objs))()
    for i, o in enumerate(objs):
        arr[i] = o.handle.value
    return arr


def steady_workspace_size(material: Material, geoms: Sequence[Geometry], n_particles, cfg: SteadyConfig,
                          grad: bool = False, n_dirs: int = 0) -> int:
    n = np.ascontiguousarray(np.asarray(n_particles, dtype=np.uint64))
    p = steady_params(cfg, n)
    b = C.c_size_t(0)
    L.check(L.load().mcbte_steady_workspace_size(material.handle, _handles(geoms), len(geoms), C.byref(p),
                                                 int(grad), int(n_dirs), C.byref(b)))
    return int(b.value)


def run_steady(material: Material, geoms: Sequence[Geometry], n_particles, cfg: SteadyConfig, *,
               out: Optional[SteadyOutputs] = None, per_particle: bool = False, workspace=None,
               stream=None) -> SteadyOutputs:
    """``mcbte_run_steady`` with device outputs (asynchronous on `stream`)."""
    n = np.ascontiguousarray(np.asarray(n_particles, dtype=np.uint64))
    if out is None:
        out = SteadyOutputs(len(geoms), material.n_bins, cfg.n_cells, cfg.per_bin, int(n.sum()), per_particle,
                            regions=cfg.regions, nscat=cfg.n_scat_max if cfg.nscat_curve else 0,
                            det_per_bin=cfg.det_per_bin)
    p = steady_params(cfg, n)
    o = out.struct()
    ws_ptr, ws_bytes = (None, 0) if workspace is None else (workspace.data_ptr(), workspace.numel() * workspace.element_size())
    L.check(L.load().mcbte_run_steady(material.handle, _handles(geoms), len(geoms), C.byref(p), C.byref(o),
                                      ws_ptr, ws_bytes, _stream_ptr(stream)))
    return out


def run_steady_noalloc(material: Material, geoms: Sequence[Geometry], n_particles, cfg: SteadyConfig,
                       out: SteadyOutputs, stream=None) -> SteadyOutputs:
    """``mcbte_run_steady_noalloc``: the steady run for callers that cannot
    allocate device memory.  `out` must already hold the device outputs; the
    library uses its fixed internal scratch and allocates nothing.  Calls
    whose GPU work overlaps race on that scratch."""
    n = np.ascontiguousarray(np.asarray(n_particles, dtype=np.uint64))
    p = steady_params(cfg, n)
    o = out.struct()
    L.check(L.load().mcbte_run_steady_noalloc(material.handle, _handles(geoms), len(geoms), C.byref(p), C.byref(o),
                                              _stream_ptr(stream)))
    return out


def run_steady_host(material: Material, geoms: Sequence[Geometry], n_particles, cfg: SteadyConfig) -> Dict:
    """``mcbte_run_steady`` with host (numpy) outputs: the library copies
    results back and synchronises before returning."""
    n = np.ascontiguousarray(np.asarray(n_particles, dtype=np.uint64))
    G, nb, nc = len(geoms), material.n_bins, cfg.n_cells
    res = {"stats": np.zeros((G, L.NSTATS))}
    if nc > 0:
        res["T"] = np.zeros((G, nc)); res["q"] = np.zeros((G, nc, 3))
    if cfg.per_bin:
        res["q_bin"] = np.zeros((G, nb))
    o = L.SteadyOut()
    o.stats = res["stats"].ctypes.data
    o.T = res["T"].ctypes.data if nc > 0 else None
    o.q = res["q"].ctypes.data if nc > 0 else None
    o.q_bin = res["q_bin"].ctypes.data if cfg.per_bin else None
    if cfg.nscat_curve:
        res["kappa_nscat"] = np.zeros((G, int(cfg.n_scat_max), 2))
        o.kappa_nscat = res["kappa_nscat"].ctypes.data
    nd = sum(int(np.prod(r[1])) for r in cfg.regions) if cfg.regions else 0
    if nd:
        res["det"] = np.zeros((nd, nb, 4) if cfg.det_per_bin else (nd, 4))
        o.det = res["det"].ctypes.data
    o.on_host = 1
    p = steady_params(cfg, n)
    st = L.load().mcbte_run_steady(material.handle, _handles(geoms), G, C.byref(p), C.byref(o), None, 0, None)
    L.check(st, allow=(L.OK, L.WARN_TRUNCATED))
    res["status"] = st
    return res


@dataclass
class TransientConfig:
    seed: int
    t_max: float
    t_meas: np.ndarray
    grid: Sequence[int]
    precision: int = L.FP32_TRACE
    max_events: int = 0
    threads_per_block: int = 0
    blocks_per_sm: int = 0
    time_budget_s: float = 0.0
    trace_events: Optional[tuple] = None
    window_times: int = 0                    # measurement times per time window (0: sized to the L2)
    regions: Sequence = ()                   # ((xmin, xmax, ymin, ymax, zmin, zmax) m, (nx, ny, nz)) per region
    time_average: bool = False               # averages over [t_{m-1}, t_m) instead of snapshots at t_m


class TransientOutputs:
    """Device outputs of a transient run: tally [n_times][nz][ny][nx][4] for the
    whole-box grid, or [n_times][n_detectors][4] when `regions` are given."""

    def __init__(self, n_times: int, grid, n_particles: int, per_particle: bool = False, device=None,
                 regions: Sequence = ()):
        import torch
        dev = device or torch.device("cuda")
        nx, ny, nz = (int(g) for g in grid)
        if regions:
            nd = sum(int(np.prod(r[1])) for r in regions)
            self.tally = torch.zeros(n_times, nd, 4, dtype=torch.float64, device=dev)
        else:
            self.tally = torch.zeros(n_times, nz, ny, nx, 4, dtype=torch.float64, device=dev)
        self.stats = torch.zeros(L.NSTATS, dtype=torch.float64, device=dev)
        self.events_pp = torch.zeros(n_particles, dtype=torch.int32, device=dev) if per_particle else None

    def struct(self):
        o = L.TransientOut()
        o.tally, o.stats, o.events_pp = _ptr(self.tally), _ptr(self.stats), _ptr(self.events_pp)
        o.on_host = 0
        return o


def transient_params(cfg: TransientConfig, n_particles: int, t_meas: np.ndarray) -> "L.TransientParams":
    p = L.TransientParams()
    p.n_particles = int(n_particles)
    p.seed = int(cfg.seed)
    p.precision = int(cfg.precision)
    p.max_events = int(cfg.max_events)
    p.t_max = float(cfg.t_max)
    p.n_times = int(t_meas.shape[0])
    p.t_meas = t_meas.ctypes.data
    p.grid[:] = [int(g) for g in cfg.grid]
    p.threads_per_block = int(cfg.threads_per_block)
    p.blocks_per_sm = int(cfg.blocks_per_sm)
    p.time_budget_s = float(cfg.time_budget_s)
    p.trace_event_start, p.trace_event_stop = _event_handles(cfg.trace_events)
    p.window_times = int(cfg.window_times)
    p.time_average = int(bool(cfg.time_average))
    regions = list(cfg.regions or ())
    if regions:
        boxes = np.ascontiguousarray([r[0] for r in regions], dtype=np.float64)
        grids = np.ascontiguousarray([r[1] for r in regions], dtype=np.int32)
        p._keep = (boxes, grids)            # host arrays read during the call
        p.n_regions, p.regions, p.region_grid = len(regions), boxes.ctypes.data, grids.ctypes.data
    return p


def run_transient(material: Material, geom: Geometry, n_particles: int, cfg: TransientConfig, *,
                  out: Optional[TransientOutputs] = None, per_particle: bool = False, workspace=None,
                  stream=None) -> TransientOutputs:
    tm = _f64(cfg.t_meas)
    if out is None:
        out = TransientOutputs(tm.shape[0], cfg.grid, n_particles, per_particle, regions=cfg.regions)
    p = transient_params(cfg, n_particles, tm)
    o = out.struct()
    ws_ptr, ws_bytes = (None, 0) if workspace is None else (workspace.data_ptr(), workspace.numel() * workspace.element_size())
    L.check(L.load().mcbte_run_transient(material.handle, geom.handle, C.byref(p), C.byref(o), ws_ptr, ws_bytes,
                                         _stream_ptr(stream)))
    return out


class GradOutputs:
    def __init__(self, n_bins: int, n_dirs: int = 0, device=None):
        import torch
        dev = device or torch.device("cuda")
        f = dict(dtype=torch.float64, device=dev)
        self.dkappa_dlogtau = torch.zeros(n_bins, **f)
        self.dkappa_dp = torch.zeros(2, **f)
        self.dkappa_dir = torch.zeros(max(n_dirs, 1), 2, **f)
        self.n_dirs = n_dirs


def grad(material: Material, geom: Geometry, n_particles: int, cfg: SteadyConfig, *, dirs=None,
         fwd: Optional[SteadyOutputs] = None, gout: Optional[GradOutputs] = None, workspace=None,
         stream=None, dp_estimator: int = L.DP_AUTO):
    """``mcbte_grad``: forward tallies plus the likelihood-ratio gradient of
    kappa with respect to per-bin log tau and the pore specularity (the
    measure-valued estimator for the latter at p = 0, 1, or wherever
    ``dp_estimator`` asks for it)."""
    import torch
    n = np.ascontiguousarray(np.asarray([n_particles], dtype=np.uint64))
    if fwd is None:
        fwd = SteadyOutputs(1, material.n_bins, cfg.n_cells, cfg.per_bin)
    nd = 0 if dirs is None else int(dirs.shape[0])
    if gout is None:
        gout = GradOutputs(material.n_bins, nd)
    dirs_t = None
    if dirs is not None:
        dirs_t = torch.as_tensor(np.asarray(dirs, dtype=np.float64)).reshape(nd, material.n_bins).to("cuda").contiguous()
    g = L.GradOut()
    g.dkappa_dlogtau = gout.dkappa_dlogtau.data_ptr()
    g.dkappa_dp = gout.dkappa_dp.data_ptr()
    g.dirs = _ptr(dirs_t)
    g.n_dirs = nd
    g.dkappa_dir = gout.dkappa_dir.data_ptr()
    g.on_host = 0
    g.dp_estimator = int(dp_estimator)
    p = steady_params(cfg, n)
    o = fwd.struct()
    ws_ptr, ws_bytes = (None, 0) if workspace is None else (workspace.data_ptr(), workspace.numel() * workspace.element_size())
    L.check(L.load().mcbte_grad(material.handle, geom.handle, C.byref(p), C.byref(o), C.byref(g), ws_ptr, ws_bytes,
                                _stream_ptr(stream)))
    if dirs_t is not None:
        gout._dirs = dirs_t     # keep alive until the stream has consumed it
    return fwd, gout
