"""C-ABI checks that need no GPU: the library loads, exports every entry
point ``include/mcbte.h`` declares, and rejects bad arguments before any
CUDA call."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from inputs import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2104_03573_gb300 import build, _lib
    build.build()
    return _lib.load()


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(mcbte_[a-z0-9_]+)\s*\(", src))
    return names


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib, n), n


def test_binding_export_list_matches_header(lib):
    from paper_2104_03573_gb300 import _lib
    assert set(_lib.EXPORTS) <= _declared()


def test_version_and_error_buffer(lib):
    from paper_2104_03573_gb300 import _lib
    assert lib.mcbte_version() == 10000
    buf = C.create_string_buffer(4)
    lib.mcbte_last_error(buf, 4)
    assert len(buf.value) <= 3


def test_geometry_validation_rejects_before_cuda(lib):
    from paper_2104_03573_gb300 import _lib, api
    bad = W.slab_z(100e-9, 300.5, 299.5)
    bad.face_type = [_lib.FACE_PERIODIC, _lib.FACE_ADIABATIC] + list(bad.face_type[2:])
    d = api.geometry_desc(bad)
    h = C.c_void_p()
    assert lib.mcbte_geometry_create(C.byref(d), C.byref(h)) == _lib.ERR_INVALID_ARG
    assert "periodic" in _lib.last_error()
    p = W.pore_lattice(100e-9, 0.25, 200e-9)
    p.pore_r = 60e-9
    assert lib.mcbte_geometry_create(C.byref(api.geometry_desc(p)), C.byref(h)) == _lib.ERR_INVALID_ARG
    g2 = W.film(10e-9)
    g2.grad_T = (1.0, float("nan"), 0.0)            # any direction, but finite
    assert lib.mcbte_geometry_create(C.byref(api.geometry_desc(g2)), C.byref(h)) == _lib.ERR_INVALID_ARG
    g3 = W.film(10e-9, p=1.5)
    assert lib.mcbte_geometry_create(C.byref(api.geometry_desc(g3)), C.byref(h)) == _lib.ERR_INVALID_ARG


def test_internal_wall_validation_rejects_before_cuda(lib):
    from paper_2104_03573_gb300 import _lib, api
    from inputs import workloads as W
    h = C.c_void_p()
    for mutate in ("outside", "normal", "spec", "count", "empty"):
        g = W.nanomesh()
        if mutate == "outside":
            g.inner = [list(s) for s in g.inner]
            g.inner[0][2] = 40e-9
        elif mutate == "normal":
            g.inner_n = [list(n) for n in g.inner_n]
            g.inner_n[1] = [0.9, 0.0]
        elif mutate == "spec":
            g.inner_p = [0.0, 1.5, 0.0, 0.0]
        elif mutate == "empty":
            g.inner = [list(s) for s in g.inner]
            g.inner[2] = [g.inner[2][0], g.inner[2][1], g.inner[2][0], g.inner[2][1]]
        d = api.geometry_desc(g)
        if mutate == "count":
            d.n_inner = 17
        assert lib.mcbte_geometry_create(C.byref(d), C.byref(h)) == _lib.ERR_INVALID_ARG, mutate


def test_material_validation_rejects_before_cuda(lib):
    from paper_2104_03573_gb300 import _lib
    n = 3
    om = np.array([1e12, 2e12, 3e12]); v = np.array([1e3, -1.0, 2e3]); tau = np.ones(3) * 1e-11
    Cc = np.ones(3)
    d = _lib.MaterialDesc()
    d.n_bins = n
    d.omega, d.v, d.tau, d.C = om.ctypes.data, v.ctypes.data, tau.ctypes.data, Cc.ctypes.data
    h = C.c_void_p()
    assert lib.mcbte_material_create(C.byref(d), C.byref(h)) == _lib.ERR_INVALID_ARG
    d.n_bins = 0
    assert lib.mcbte_material_create(C.byref(d), C.byref(h)) == _lib.ERR_INVALID_ARG
    d.n_bins = n
    d.C = None
    assert lib.mcbte_material_create(C.byref(d), C.byref(h)) == _lib.ERR_INVALID_ARG
    # two-phonon times must be > 0 (+inf allowed)
    v[1] = 1.5e3
    d.C = Cc.ctypes.data
    bad_imp = np.array([1e-12, np.inf, 0.0])
    d.tau_imp = bad_imp.ctypes.data
    assert lib.mcbte_material_create(C.byref(d), C.byref(h)) == _lib.ERR_INVALID_ARG
    bad_imp[2] = -1.0
    assert lib.mcbte_material_create(C.byref(d), C.byref(h)) == _lib.ERR_INVALID_ARG
    bad_imp[2] = np.nan
    assert lib.mcbte_material_create(C.byref(d), C.byref(h)) == _lib.ERR_INVALID_ARG


def test_null_arguments_rejected(lib):
    from paper_2104_03573_gb300 import _lib
    h = C.c_void_p()
    assert lib.mcbte_material_create(None, C.byref(h)) == _lib.ERR_INVALID_ARG
    assert lib.mcbte_geometry_create(None, C.byref(h)) == _lib.ERR_INVALID_ARG
    assert lib.mcbte_run_steady(None, None, 1, None, None, None, 0, None) == _lib.ERR_INVALID_ARG
    assert lib.mcbte_run_transient(None, None, None, None, None, 0, None) == _lib.ERR_INVALID_ARG
    assert lib.mcbte_grad(None, None, None, None, None, None, 0, None) == _lib.ERR_INVALID_ARG


def test_product_package_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_2104_03573_gb300")
    for root, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(root, f)).read()
                assert "oracle" not in src.lower().replace("oracle-free", ""), f


def test_bench_l2_probe_builds_apart_and_rejects_bad_sizes_before_cuda(lib):
    import bench
    probe = bench.load_probe()
    assert probe.bench_l2_reduction_probe(None, 16, 10, None) == 1
    assert probe.bench_l2_reduction_probe(C.c_void_p(256), 6, 10, None) == 1
    assert probe.bench_l2_reduction_probe(C.c_void_p(256), 0, 10, None) == 1
    assert not hasattr(lib, "mcbte_l2_reduction_probe")      # a measurement of the bench, not a library call
