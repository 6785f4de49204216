"""Oracle for the deviational Monte Carlo LBTE solver (arXiv:2104.03573).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the product package.
It shares no code with the CUDA library.

``mcbte_oracle.cpp`` is a plain FP64 scalar tracer (one particle after the
other, ``std::thread`` over contiguous particle ranges).  This module loads
it with ctypes and turns its raw sums into physical tallies exactly as the
paper's estimators define them:

* steady temperature  T_dev = (E'_eff / (C V)) sum_i s_i l_i / V_g,i   (Eq. temp_steady)
* steady flux         q_x   = (E'_eff / V) sum_i s_i l_x,i              (Eq. flux_x_steady)
* transient snapshots T = s E_eff / (C V), q_x = s E_eff V_g,x / V     (Eq. sampling, Sec. 3.4)
* E_eff = E_tot / N, E'_eff = E'_tot / N                                (Sec. 3.1, Eq. dev_steady_rate)

``closed_forms.py`` holds the deterministic solutions the oracle is pinned
against.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mcbte_oracle.cpp")
_LIB = os.path.join(_HERE, "libmcbte_oracle.so")

# indices into or_out.scal
SUMX, SUMX2, EVENTS, TRUNC, ABSORBED, SIGNED_ABS, SIGNED_EMIT, RSUM, GP, GP2, ETOT, CTOT, VSOLID, MAXEV = range(14)


class _Params(C.Structure):
    _fields_ = [
        ("n_bins", C.c_int), ("omega", C.c_void_p), ("v", C.c_void_p), ("tau", C.c_void_p),
        ("C", C.c_void_p), ("D", C.c_void_p), ("domega", C.c_void_p), ("T_lin", C.c_double),
        ("tau_imp", C.c_void_p), ("spec_bin", C.c_void_p),
        ("L", C.c_double * 3), ("face_type", C.c_int * 6), ("face_T", C.c_double * 6),
        ("face_p", C.c_double * 6), ("T_eq", C.c_double), ("grad_T", C.c_double * 3),
        ("pore", C.c_int), ("pore_c", C.c_double * 2), ("pore_r", C.c_double), ("pore_p", C.c_double),
        ("gauss", C.c_int), ("gauss_c", C.c_double * 3), ("gauss_sigma", C.c_double),
        ("gauss_dT", C.c_double),
        ("n_inner", C.c_int), ("inner", (C.c_double * 4) * 16), ("inner_n", (C.c_double * 2) * 16),
        ("inner_p", C.c_double * 16),
        ("seed", C.c_uint64), ("batch_index", C.c_uint32), ("transient", C.c_int),
        ("n_particles", C.c_uint64), ("pid_begin", C.c_uint64), ("pid_end", C.c_uint64),
        ("n_scat_max", C.c_int), ("max_events", C.c_uint64),
        ("n_cells", C.c_int), ("cell_axis", C.c_int), ("tally_axis", C.c_int),
        ("t_max", C.c_double), ("n_times", C.c_int), ("t_meas", C.c_void_p), ("grid", C.c_int * 3),
        ("n_regions", C.c_int), ("regions", C.c_void_p), ("region_grid", C.c_void_p), ("time_average", C.c_int),
        ("det_per_bin", C.c_int),
        ("nscat_curve", C.c_int), ("want_grad", C.c_int), ("dp_mvd", C.c_int), ("n_dirs", C.c_int), ("dirs", C.c_void_p), ("n_threads", C.c_int),
    ]


class _Out(C.Structure):
    _fields_ = [
        ("T_sum", C.c_void_p), ("Q_sum", C.c_void_p), ("qbin_sum", C.c_void_p), ("snap", C.c_void_p),
        ("events_pp", C.c_void_p), ("X_pp", C.c_void_p), ("G", C.c_void_p),
        ("dir_sum", C.c_void_p), ("dir_sum2", C.c_void_p), ("curve", C.c_void_p), ("scal", C.c_double * 16),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with the system C++ compiler (no FMA contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-pthread", _SRC, "-o", _LIB + ".tmp"]
    subprocess.check_call(cmd)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        L.or_run.argtypes = [C.POINTER(_Params), C.POINTER(_Out)]
        L.or_run.restype = C.c_int
        L.or_tables.argtypes = [C.POINTER(_Params)] + [C.c_void_p] * 5
        L.or_tables.restype = C.c_int
        L.or_sources.argtypes = [C.POINTER(_Params), C.c_void_p, C.POINTER(C.c_int)]
        L.or_sources.restype = C.c_int
        L.or_first_hit.argtypes = [C.POINTER(_Params), C.c_void_p, C.c_void_p,
                                   C.POINTER(C.c_double), C.POINTER(C.c_int)]
        L.or_philox.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.or_dEdT.argtypes = [C.c_double, C.c_double]
        L.or_dEdT.restype = C.c_double
        L.or_log.argtypes = [C.c_double]
        L.or_log.restype = C.c_double
        L.or_sincos2pi.argtypes = [C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.or_alias.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.or_alias_draw.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_uint32, C.c_uint32, C.c_uint32]
        L.or_alias_draw.restype = C.c_int
        L.or_set_libm.argtypes = [C.c_int]
        L.or_set_libm.restype = None
        _lib = L
    return _lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data


def _f64(a) -> Optional[np.ndarray]:
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


class _Keep:
    """Holds numpy buffers alive while a ctypes call uses their pointers."""

    def __init__(self):
        self.items = []

    def add(self, a):
        self.items.append(a)
        return a


def _set_inner(P, geom) -> None:
    inner = list(getattr(geom, "inner", ()) or ())
    if len(inner) > 16:
        raise ValueError("at most 16 internal boundaries")
    P.n_inner = len(inner)
    for k, seg in enumerate(inner):
        P.inner[k][:] = [float(c) for c in seg]
        P.inner_n[k][:] = [float(c) for c in geom.inner_n[k]]
        P.inner_p[k] = float(geom.inner_p[k])


def _params(material, geom, keep: _Keep, **kw) -> _Params:
    P = _Params()
    P.n_bins = material.n_bins
    om, v, tau = (keep.add(_f64(material.omega)), keep.add(_f64(material.v)), keep.add(_f64(material.tau)))
    P.omega, P.v, P.tau = _ptr(om), _ptr(v), _ptr(tau)
    if material.C is not None:
        P.C = _ptr(keep.add(_f64(material.C)))
    else:
        P.D = _ptr(keep.add(_f64(material.D)))
        P.domega = _ptr(keep.add(_f64(material.domega)))
    P.T_lin = material.T_lin
    if getattr(material, "tau_imp", None) is not None:
        P.tau_imp = _ptr(keep.add(_f64(material.tau_imp)))
    if getattr(material, "spec_bin", None) is not None:
        P.spec_bin = _ptr(keep.add(_f64(material.spec_bin)))
    if geom is not None:
        P.L[:] = [float(x) for x in geom.L]
        P.face_type[:] = [int(x) for x in geom.face_type]
        P.face_T[:] = [float(x) for x in geom.face_T]
        P.face_p[:] = [float(x) for x in geom.face_p]
        P.T_eq = geom.T_eq
        P.grad_T[:] = [float(x) for x in geom.grad_T]
        P.pore = int(geom.pore)
        P.pore_c[:] = [float(x) for x in geom.pore_c]
        P.pore_r = geom.pore_r
        P.pore_p = geom.pore_p
        P.gauss = int(geom.gauss)
        P.gauss_c[:] = [float(x) for x in geom.gauss_c]
        P.gauss_sigma = geom.gauss_sigma
        P.gauss_dT = geom.gauss_dT
        _set_inner(P, geom)
    for k, val in kw.items():
        setattr(P, k, val)
    return P


class libm_mode:
    """Context manager: inside it the tracer evaluates ln, sin and cos with
    the C library instead of its fixed series (shows what that choice
    changes per particle; the default series mode is the reference)."""

    def __enter__(self):
        lib().or_set_libm(1)
        return self

    def __exit__(self, *exc):
        lib().or_set_libm(0)
        return False


def philox(ctr: Sequence[int], key: Sequence[int]) -> np.ndarray:
    c = np.array(ctr, dtype=np.uint32)
    k = np.array(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().or_philox(c.ctypes.data, k.ctypes.data, o.ctypes.data)
    return o


def dEdT(omega: float, T: float) -> float:
    return lib().or_dEdT(float(omega), float(T))


def series_log(x: float) -> float:
    return lib().or_log(float(x))


def series_sincos2pi(r: float):
    s, c = C.c_double(0), C.c_double(0)
    lib().or_sincos2pi(float(r), C.byref(s), C.byref(c))
    return s.value, c.value


def alias_table(w: np.ndarray):
    w = _f64(w)
    n = w.shape[0]
    prob = np.zeros(n); thr = np.zeros(n, dtype=np.uint64); al = np.zeros(n, dtype=np.int32)
    lib().or_alias(n, w.ctypes.data, prob.ctypes.data, thr.ctypes.data, al.ctypes.data)
    return prob, thr, al


def alias_draw(thr: np.ndarray, al: np.ndarray, wcol: int, lo: int, hi: int) -> int:
    return lib().or_alias_draw(thr.shape[0], thr.ctypes.data, al.ctypes.data, wcol, lo, hi)


def tables(material) -> dict:
    keep = _Keep()
    P = _params(material, None, keep)
    n = material.n_bins
    Cb = np.zeros(n); prob = np.zeros(3 * n); thr = np.zeros(3 * n, dtype=np.uint64)
    al = np.zeros(3 * n, dtype=np.int32); sums = np.zeros(3)
    rc = lib().or_tables(C.byref(P), Cb.ctypes.data, prob.ctypes.data, thr.ctypes.data,
                         al.ctypes.data, sums.ctypes.data)
    if rc:
        raise ValueError(f"oracle table build failed ({rc})")
    return {"C": Cb, "prob": prob.reshape(3, n), "thr": thr.reshape(3, n), "alias": al.reshape(3, n),
            "C_tot": sums[0], "sum_Cv": sums[1], "sum_C_over_tau": sums[2]}


def sources(material, geom, transient: bool = False, t_max: float = 0.0) -> dict:
    keep = _Keep()
    P = _params(material, geom, keep, transient=int(transient), t_max=t_max)
    out = np.zeros(16)
    ns = C.c_int(0)
    rc = lib().or_sources(C.byref(P), out.ctypes.data, C.byref(ns))
    if rc:
        raise ValueError(f"oracle source setup failed ({rc})")
    return {"E_tot": out[0], "V_solid": out[1], "E": out[2:2 + ns.value].copy()}


def first_hit(geom, x_nm, u):
    keep = _Keep()
    from inputs.workloads import gray
    P = _params(gray(1.0, 1.0), geom, keep)
    x = _f64(x_nm); uu = _f64(u)
    d = C.c_double(0); f = C.c_int(0)
    lib().or_first_hit(C.byref(P), x.ctypes.data, uu.ctypes.data, C.byref(d), C.byref(f))
    return d.value, f.value


def dir_about_vector(gv, sgn: float, mu: float, wphi: int) -> np.ndarray:
    """Body-particle direction with polar cosine mu about sgn * gv (unit)."""
    g = _f64(gv)
    u = np.zeros(3)
    f = lib().or_dir_about_vector
    f.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_uint32, C.c_void_p]
    f.restype = C.c_int
    f(g.ctypes.data, float(sgn), float(mu), int(wphi), u.ctypes.data)
    return u


def in_hole(geom, x_nm: float, y_nm: float) -> bool:
    """True if (x, y) in nm lies inside a hole bounded by the internal walls."""
    keep = _Keep()
    from inputs.workloads import gray
    P = _params(gray(1.0, 1.0), geom, keep)
    f = lib().or_in_hole
    f.argtypes = [C.c_void_p, C.c_double, C.c_double]
    f.restype = C.c_int
    return bool(f(C.byref(P), float(x_nm), float(y_nm)))


def _kappa_gradient(geom, axis: int) -> float:
    """dT/dx along `axis` that defines kappa_eff = -q / (dT/dx): the control
    gradient if one is set, else the isothermal wall difference over L."""
    g = float(geom.grad_T[axis])
    if g != 0.0:
        return g
    lo = {0: 3, 1: 0, 2: 4}[axis]
    hi = {0: 1, 1: 2, 2: 5}[axis]
    if geom.face_type[lo] == 0 and geom.face_type[hi] == 0:
        return (geom.face_T[hi] - geom.face_T[lo]) / geom.L[axis]
    return float("nan")


def dp_mvd(geom, dp_estimator: int = 0) -> bool:
    """Whether d kappa / d p_pore takes the measure-valued estimator."""
    if not getattr(geom, "pore", False):
        return False
    p = float(geom.pore_p)
    return dp_estimator == 2 or (dp_estimator == 0 and (p <= 0.0 or p >= 1.0))


def run_steady(material, geom, run, *, pid_begin: int = 0, pid_end: Optional[int] = None,
               per_particle: bool = False, grad: bool = False, dirs: Optional[np.ndarray] = None,
               n_threads: int = 0, batch_index: int = 0, n_total: Optional[int] = None,
               dp_estimator: int = 0, nscat_curve: bool = False, det_per_bin: bool = False) -> dict:
    """Trace particles [pid_begin, pid_end) of a steady run of N = run.n (or
    n_total) particles and return raw sums plus the physical tallies.

    dp_estimator selects the estimator of d kappa / d p_pore when grad is set:
    1 the likelihood ratio of the specular / diffuse draw, 2 the measure-valued
    one (each particle's phantom trace with one pore hit's branch flipped),
    0 the likelihood ratio for 0 < p < 1 and the measure-valued one at p = 0, 1.
    nscat_curve adds "kappa_nscat" [n_scat_max][2]: kappa and its standard
    error for every N_scat_max' = 1..n_scat_max, from the same trajectories.
    det_per_bin splits the detector-region outputs by frequency bin
    (det_T [n_det][n_bins], det_q [n_det][n_bins][3])."""
    N = int(n_total if n_total is not None else run.n)
    pe = N if pid_end is None else int(pid_end)
    keep = _Keep()
    n = material.n_bins
    dirs_a = None
    if grad and dirs is not None:
        dirs_a = keep.add(np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1, n))
    P = _params(material, geom, keep, seed=int(run.seed), batch_index=int(batch_index), transient=0,
                n_particles=N, pid_begin=int(pid_begin), pid_end=pe, n_scat_max=int(run.n_scat_max),
                max_events=int(run.max_events), n_cells=int(run.n_cells), cell_axis=int(run.cell_axis),
                tally_axis=int(run.tally_axis), want_grad=int(grad),
                dp_mvd=int(bool(grad) and dp_mvd(geom, dp_estimator)), nscat_curve=int(bool(nscat_curve)),
                n_dirs=0 if dirs_a is None else dirs_a.shape[0],
                dirs=_ptr(dirs_a), n_threads=int(n_threads))
    npp = pe - int(pid_begin)
    nc = int(run.n_cells)
    T = np.zeros(max(nc, 1)); Q = np.zeros((max(nc, 1), 3)); qb = np.zeros(n)
    ev = np.zeros(npp, dtype=np.uint32) if per_particle else None
    Xp = np.zeros(npp) if per_particle else None
    G = np.zeros(n) if grad else None
    nd = 0 if dirs_a is None else dirs_a.shape[0]
    ds = np.zeros(max(nd, 1)); ds2 = np.zeros(max(nd, 1))
    O = _Out()
    O.T_sum = T.ctypes.data if nc > 0 else None
    O.Q_sum = Q.ctypes.data if nc > 0 else None
    O.qbin_sum = qb.ctypes.data
    O.events_pp = _ptr(ev); O.X_pp = _ptr(Xp); O.G = _ptr(G)
    O.dir_sum = ds.ctypes.data if nd else None
    O.dir_sum2 = ds2.ctypes.data if nd else None
    curve = np.zeros((max(int(run.n_scat_max), 1), 2)) if nscat_curve else None
    O.curve = _ptr(curve)
    regions = list(getattr(run, "regions", ()) or ())
    det = None
    if regions:
        boxes = keep.add(np.ascontiguousarray([rg[0] for rg in regions], dtype=np.float64))
        grids = keep.add(np.ascontiguousarray([rg[1] for rg in regions], dtype=np.int32))
        P.n_regions, P.regions, P.region_grid = len(regions), boxes.ctypes.data, grids.ctypes.data
        P.det_per_bin = int(bool(det_per_bin))
        nd_ = int(sum(int(np.prod(rg[1])) for rg in regions))
        det = np.zeros((nd_, n, 4) if det_per_bin else (nd_, 4))
        O.snap = det.ctypes.data
    rc = lib().or_run(C.byref(P), C.byref(O))
    if rc:
        raise ValueError(f"oracle run failed ({rc})")
    sc = np.array(O.scal[:])
    r = {"raw_T": T[:nc], "raw_Q": Q[:nc], "raw_qbin": qb, "scal": sc, "events_pp": ev, "X_pp": Xp,
         "N": N, "n_traced": npp}
    if regions:
        v_det = np.concatenate([np.full(int(np.prod(rg[1])),
                                        np.prod(np.asarray(rg[0])[1::2] - np.asarray(rg[0])[0::2]) / np.prod(rg[1]))
                                for rg in regions])
        r["det_raw"] = det
        r["det_V"] = v_det
    E_tot, C_tot, V = sc[ETOT], sc[CTOT], sc[VSOLID]
    E_eff = E_tot / N
    Vbox = float(geom.L[0] * geom.L[1] * geom.L[2])
    if nc > 0:
        Vc = Vbox / nc
        r["T"] = (E_eff / (C_tot * Vc)) * T[:nc] * 1e-12
        r["q"] = (E_eff / Vc) * Q[:nc] * 1e-9
    r["q_bin"] = (E_eff / V) * qb * 1e-9
    if regions:
        vol = r["det_V"][:, None] if det_per_bin else r["det_V"]
        r["det_T"] = (E_eff / (C_tot * vol)) * det[..., 0] * 1e-12
        r["det_q"] = (E_eff / vol)[..., None] * det[..., 1:] * 1e-9
    sx, sx2 = sc[SUMX], sc[SUMX2]
    mean = sx / npp if npp else 0.0
    var = (sx2 - npp * mean * mean) / (npp - 1) if npp > 1 else 0.0
    r["q_mean"] = (E_eff / V) * sx * 1e-9
    r["q_se"] = (E_tot / V) * 1e-9 * math.sqrt(max(var, 0.0) / npp) * (npp / N) if npp else 0.0
    gk = _kappa_gradient(geom, run.tally_axis)
    r["grad_eff"] = gk
    r["kappa"] = -r["q_mean"] / gk
    r["kappa_se"] = r["q_se"] / abs(gk)
    r["kappa_cell"] = r["kappa"] * V / Vbox
    if nscat_curve:
        cm = curve[:, 0] / npp
        cv = (curve[:, 1] - npp * cm * cm) / max(npp - 1, 1)
        r["raw_curve"] = curve
        r["kappa_nscat"] = np.stack([-((E_eff / V) * curve[:, 0] * 1e-9) / gk,
                                     (E_tot / V) * 1e-9 * np.sqrt(np.maximum(cv, 0.0) / npp) * (npp / N) / abs(gk)],
                                    axis=1)
    r["events"] = sc[EVENTS]
    r["truncated"] = sc[TRUNC]
    r["E_tot"] = E_tot
    r["C_tot"] = C_tot
    r["V_solid"] = V
    if grad:
        tb = tables(material)
        w = tb["C"] / np.asarray(material.tau, dtype=np.float64)
        pi = w / w.sum()
        scale = -(E_eff / V) * 1e-9 / gk
        r["raw_G"] = G
        r["dkappa_dlogtau"] = scale * (G + sc[RSUM] * pi)
        gp_mean = sc[GP] / npp
        gp_var = (sc[GP2] - npp * gp_mean * gp_mean) / max(npp - 1, 1)
        r["dkappa_dp"] = scale * sc[GP]
        r["dkappa_dp_se"] = abs(scale) * math.sqrt(max(gp_var, 0.0) * npp)
        if nd:
            dm = ds[:nd] / npp
            dv = (ds2[:nd] - npp * dm * dm) / max(npp - 1, 1)
            r["dkappa_dir"] = scale * ds[:nd]
            r["dkappa_dir_se"] = abs(scale) * np.sqrt(np.maximum(dv, 0.0) * npp)
    return r


def run_transient(material, geom, run, *, pid_begin: int = 0, pid_end: Optional[int] = None,
                  per_particle: bool = False, n_threads: int = 0, n_total: Optional[int] = None) -> dict:
    N = int(n_total if n_total is not None else run.n)
    pe = N if pid_end is None else int(pid_end)
    keep = _Keep()
    t_meas = keep.add(_f64(run.t_meas))
    nx, ny, nz = (int(g) for g in run.grid)
    P = _params(material, geom, keep, seed=int(run.seed), transient=1, n_particles=N,
                pid_begin=int(pid_begin), pid_end=pe, n_scat_max=0, max_events=int(run.max_events),
                t_max=float(run.t_max), n_times=int(t_meas.shape[0]), t_meas=t_meas.ctypes.data,
                tally_axis=2, n_threads=int(n_threads))
    P.grid[:] = [nx, ny, nz]
    P.time_average = int(bool(getattr(run, "time_average", False)))
    nt = t_meas.shape[0]
    regions = list(getattr(run, "regions", ()) or ())
    if regions:
        boxes = keep.add(np.ascontiguousarray([r[0] for r in regions], dtype=np.float64))
        grids = keep.add(np.ascontiguousarray([r[1] for r in regions], dtype=np.int32))
        P.n_regions, P.regions, P.region_grid = len(regions), boxes.ctypes.data, grids.ctypes.data
        n_det = int(sum(int(np.prod(r[1])) for r in regions))
        snap = np.zeros((nt, n_det, 4))
        v_det = np.concatenate([np.full(int(np.prod(r[1])),
                                        np.prod(np.asarray(r[0])[1::2] - np.asarray(r[0])[0::2]) / np.prod(r[1]))
                                for r in regions])
    else:
        snap = np.zeros((nt, nz, ny, nx, 4))
        v_det = float(geom.L[0] * geom.L[1] * geom.L[2]) / (nx * ny * nz)
    npp = pe - int(pid_begin)
    ev = np.zeros(npp, dtype=np.uint32) if per_particle else None
    O = _Out()
    O.snap = snap.ctypes.data
    O.events_pp = _ptr(ev)
    rc = lib().or_run(C.byref(P), C.byref(O))
    if rc:
        raise ValueError(f"oracle run failed ({rc})")
    sc = np.array(O.scal[:])
    E_eff = sc[ETOT] / N
    Vc = v_det if regions else np.float64(v_det)
    vb = Vc[None, :] if regions else Vc
    out = np.empty_like(snap)
    out[..., 0] = (E_eff / (sc[CTOT] * vb)) * snap[..., 0]
    out[..., 1:] = (E_eff / vb)[..., None] * snap[..., 1:] * 1e3 if regions else (E_eff / vb) * snap[..., 1:] * 1e3
    return {"raw": snap, "tally": out, "scal": sc, "events_pp": ev, "events": sc[EVENTS],
            "E_tot": sc[ETOT], "C_tot": sc[CTOT], "N": N, "V_cell": Vc}
