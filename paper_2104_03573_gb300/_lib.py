"""ctypes view of ``include/mcbte.h``: structure layouts and the loaded
library.  Argument marshalling only; every step of the method runs in the
CUDA library.  Loading fails loudly when the library has not been built."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmcbte.so")

OK, ERR_INVALID_ARG, ERR_CUDA, ERR_OOM, ERR_TIMEOUT, WARN_TRUNCATED, ERR_WORKSPACE, ERR_REPLAY = range(8)
FACE_ISOTHERMAL, FACE_ADIABATIC, FACE_PERIODIC = 0, 1, 2
FP64_PLAIN, FP32_TRACE = 0, 1
DP_AUTO, DP_LIKELIHOOD_RATIO, DP_MEASURE_VALUED = 0, 1, 2
(STAT_KAPPA, STAT_KAPPA_SE, STAT_Q_MEAN, STAT_Q_SE, STAT_SUMX, STAT_SUMX2, STAT_EVENTS, STAT_TRUNCATED,
 STAT_E_TOT, STAT_MAX_EVENTS, STAT_KAPPA_CELL, STAT_SIGNED_EMITTED, STAT_SIGNED_ABSORBED, STAT_STATUS,
 STAT_N, STAT_ABSORBED) = range(16)
NSTATS = 16

EXPORTS = [
    "mcbte_last_error", "mcbte_version", "mcbte_material_create", "mcbte_material_destroy",
    "mcbte_material_n_bins", "mcbte_material_tables", "mcbte_geometry_create", "mcbte_geometry_destroy",
    "mcbte_steady_workspace_size", "mcbte_run_steady", "mcbte_transient_workspace_size",
    "mcbte_run_transient", "mcbte_grad", "mcbte_run_steady_noalloc",
]


class MaterialDesc(C.Structure):
    _fields_ = [("n_bins", C.c_int), ("omega", C.c_void_p), ("v", C.c_void_p), ("tau", C.c_void_p),
                ("C", C.c_void_p), ("D", C.c_void_p), ("domega", C.c_void_p), ("T_lin", C.c_double),
                ("spec_bin", C.c_void_p), ("tau_imp", C.c_void_p)]


class GeometryDesc(C.Structure):
    _fields_ = [("L", C.c_double * 3), ("face_type", C.c_int * 6), ("face_T", C.c_double * 6),
                ("face_p", C.c_double * 6), ("T_eq", C.c_double), ("grad_T", C.c_double * 3),
                ("pore", C.c_int), ("pore_c", C.c_double * 2), ("pore_r", C.c_double), ("pore_p", C.c_double),
                ("gauss", C.c_int), ("gauss_c", C.c_double * 3), ("gauss_sigma", C.c_double),
                ("gauss_dT", C.c_double), ("n_inner", C.c_int), ("inner", (C.c_double * 4) * 16),
                ("inner_n", (C.c_double * 2) * 16), ("inner_p", C.c_double * 16)]


class SteadyParams(C.Structure):
    _fields_ = [("n_particles", C.c_void_p), ("seed", C.c_uint64), ("precision", C.c_int),
                ("n_scat_max", C.c_int), ("max_events", C.c_uint64), ("n_cells", C.c_int),
                ("cell_axis", C.c_int), ("tally_axis", C.c_int), ("per_bin", C.c_int),
                ("threads_per_block", C.c_int), ("blocks_per_sm", C.c_int), ("time_budget_s", C.c_double),
                ("trace_event_start", C.c_void_p), ("trace_event_stop", C.c_void_p),
                ("seed_device", C.c_void_p), ("refill_threshold", C.c_int), ("cell_flux_axis", C.c_int),
                ("n_regions", C.c_int), ("regions", C.c_void_p), ("region_grid", C.c_void_p),
                ("nscat_curve", C.c_int), ("det_per_bin", C.c_int), ("tail_lanes", C.c_int),
                ("pid_begin", C.c_void_p), ("n_total", C.c_void_p)]


class SteadyOut(C.Structure):
    _fields_ = [("T", C.c_void_p), ("q", C.c_void_p), ("q_bin", C.c_void_p), ("stats", C.c_void_p),
                ("events_pp", C.c_void_p), ("X_pp", C.c_void_p), ("on_host", C.c_int), ("det", C.c_void_p),
                ("kappa_nscat", C.c_void_p)]


class TransientParams(C.Structure):
    _fields_ = [("n_particles", C.c_uint64), ("seed", C.c_uint64), ("precision", C.c_int),
                ("max_events", C.c_uint64), ("t_max", C.c_double), ("n_times", C.c_int),
                ("t_meas", C.c_void_p), ("grid", C.c_int * 3), ("threads_per_block", C.c_int),
                ("blocks_per_sm", C.c_int), ("time_budget_s", C.c_double),
                ("trace_event_start", C.c_void_p), ("trace_event_stop", C.c_void_p), ("window_times", C.c_int),
                ("n_regions", C.c_int), ("regions", C.c_void_p), ("region_grid", C.c_void_p),
                ("time_average", C.c_int)]


class TransientOut(C.Structure):
    _fields_ = [("tally", C.c_void_p), ("stats", C.c_void_p), ("events_pp", C.c_void_p), ("on_host", C.c_int)]


class GradOut(C.Structure):
    _fields_ = [("dkappa_dlogtau", C.c_void_p), ("dkappa_dp", C.c_void_p), ("dirs", C.c_void_p),
                ("n_dirs", C.c_int), ("dkappa_dir", C.c_void_p), ("on_host", C.c_int),
                ("dp_estimator", C.c_int)]


_lib = None


def load(path: str = LIB_PATH):
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"MCBTE CUDA library not built: {path} is missing "
                           "(run paper_2104_03573_gb300.build.build())")
    L = C.CDLL(path)
    vp = C.c_void_p
    L.mcbte_last_error.argtypes = [C.c_char_p, C.c_size_t]
    L.mcbte_last_error.restype = C.c_int
    L.mcbte_version.restype = C.c_int
    L.mcbte_material_create.argtypes = [C.POINTER(MaterialDesc), C.POINTER(vp)]
    L.mcbte_material_destroy.argtypes = [vp]
    L.mcbte_material_n_bins.argtypes = [vp]
    L.mcbte_material_tables.argtypes = [vp, vp, vp, vp, vp, vp]
    L.mcbte_geometry_create.argtypes = [C.POINTER(GeometryDesc), C.POINTER(vp)]
    L.mcbte_geometry_destroy.argtypes = [vp]
    L.mcbte_steady_workspace_size.argtypes = [vp, vp, C.c_int, C.POINTER(SteadyParams), C.c_int, C.c_int,
                                              C.POINTER(C.c_size_t)]
    L.mcbte_run_steady.argtypes = [vp, vp, C.c_int, C.POINTER(SteadyParams), C.POINTER(SteadyOut), vp,
                                   C.c_size_t, vp]
    L.mcbte_transient_workspace_size.argtypes = [vp, vp, C.POINTER(TransientParams), C.POINTER(C.c_size_t)]
    L.mcbte_run_transient.argtypes = [vp, vp, C.POINTER(TransientParams), C.POINTER(TransientOut), vp,
                                      C.c_size_t, vp]
    L.mcbte_grad.argtypes = [vp, vp, C.POINTER(SteadyParams), C.POINTER(SteadyOut), C.POINTER(GradOut), vp,
                             C.c_size_t, vp]
    L.mcbte_run_steady_noalloc.argtypes = [vp, vp, C.c_int, C.POINTER(SteadyParams), C.POINTER(SteadyOut), vp]
    for name in ("mcbte_material_create", "mcbte_material_tables", "mcbte_geometry_create",
                 "mcbte_steady_workspace_size", "mcbte_run_steady", "mcbte_transient_workspace_size",
                 "mcbte_run_transient", "mcbte_grad", "mcbte_run_steady_noalloc"):
        getattr(L, name).restype = C.c_int
    _lib = L
    return L


def last_error() -> str:
    buf = C.create_string_buffer(1024)
    load().mcbte_last_error(buf, 1024)
    return buf.value.decode(errors="replace")


class MCBTEError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"mcbte status {status}: {msg}")
        self.status = status


def check(status: int, allow=(OK,)):
    if status not in allow:
        raise MCBTEError(status, last_error())
    return status
