"""Build the MCBTE CUDA library in-tree for sm_103a (GB300).

Translation units are compiled in parallel with nvcc and linked into
``paper_2104_03573_gb300/libmcbte.so``.  The FP64 parts (table build, run
setup, FP64 tracers, finalisation) are compiled with ``--fmad=false`` so
every floating-point operation is the one written (bitwise-reproducible
against a CPU implementation of the same arithmetic); the FP32 tracers keep
fused multiply-adds.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libmcbte.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

# (source, extra flags, fused multiply-add allowed)
UNITS = [
    ("tables.cu", [], False),
    ("setup.cu", [], False),
    ("api.cu", [], False),
    ("tracer_steady.cu", ["-DMCBTE_F64=1"], False),
    ("tracer_steady.cu", ["-DMCBTE_F32=1", "-DMCBTE_F32_PART=0"], True),
    ("tracer_steady.cu", ["-DMCBTE_F32=1", "-DMCBTE_F32_PART=1"], True),
    ("tracer_transient.cu", ["-DMCBTE_F64=1"], False),
    ("tracer_transient.cu", ["-DMCBTE_F32=1"], True),
]


def _nvcc() -> str:
    p = shutil.which("nvcc")
    if p:
        return p
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found")


def _sources_mtime() -> float:
    m = 0.0
    for root in (CSRC, os.path.join(os.path.dirname(HERE), "include")):
        for f in os.listdir(root):
            m = max(m, os.path.getmtime(os.path.join(root, f)))
    return m


def build(force: bool = False, verbose: bool = False, ptxas_v: bool = False) -> str:
    units = [u for u in UNITS if os.path.exists(os.path.join(CSRC, u[0]))]
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _sources_mtime():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
                     "-I", CSRC]
    if ptxas_v:
        common += ["-Xptxas", "-v"]

    def compile_one(i_u):
        i, (src, flags, fmad) = i_u
        obj = os.path.join(BUILD, f"{i:02d}_{os.path.splitext(src)[0]}.o")
        cmd = [nvcc] + common + flags + [f"--fmad={'true' if fmad else 'false'}", "-c",
                                         os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src} {flags}:\n{r.stdout}\n{r.stderr}")
        if verbose or ptxas_v:
            sys.stderr.write(r.stdout + r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=min(len(units), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, enumerate(units)))
    tmp = LIB + ".tmp"
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_v="-v" in sys.argv))
