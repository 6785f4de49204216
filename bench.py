#!/usr/bin/env python3
"""Benchmark of the deviational Monte Carlo phonon-BTE hot path on GB300.

Default workload (`si_slab`): steady cross-plane silicon-like film, L = 1 um
(a 1 um cube, periodic x, y), BvK dispersion with 3 x 1000 bins and Holland
relaxation times at 300 K, walls at 300 +/- 0.5 K, 1e7 deviational
particles, 50 track-length cells and the frequency-resolved flux.  One step
= one full run of the hot path: run setup, tracing of all particles,
finalisation.  Our arm times the persistent FP32 tracer (FP64-exact
fixed-point tallies) and reports particle-events/s plus seconds to a 1 %
standard error on kappa_eff (t_step * (SE_rel / 0.01)^2), with the plain FP64
tracer timed beside it on the same inputs.

Other workloads (`--workload`), same line format:
  si_slab_imp    the default slab with a separate two-phonon (impurity) clock,
                 tau_imp^-1 = 2e-44 omega^4
  nanomesh       the paper's square-pore nanomesh (four internal walls), 1e6
                 particles, N_scat_max 10, separate two-phonon clock
  transient_box  2x2x1 um diffuse box, +1 K Gaussian hot spot, 1e8 particles,
                 64x64x32 cells x 200 snapshot times (fixed-point L2 reductions
                 in L2-sized time windows); also reports the reductions' rate
                 against the library's L2 reduction probe
  transient_box_avg  the same box with 200 time-bin averages instead of
                 snapshots
  film_batch     64 films 10 nm..10 um in one persistent launch replayed as
                 a CUDA graph, 1.4e8 particles in total
  pore_grad      nanoporous film, 5e7 particles, forward + likelihood-ratio
                 gradient over 3000 log-tau scales + measure-valued derivative
                 in the pore specularity at p = 0
  pore_nscat     nanoporous cell without symmetry (off-centre pore, diagonal
                 control gradient), 1e7 particles, kappa for every
                 N_scat_max = 1..32 from one run (convergence study)

`--impl reference` times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload.  Multi-GPU (torchrun): every rank traces its own
independent sample (seed offset by rank): weak scaling, no collective on the
data path.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time
from dataclasses import replace

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from inputs import workloads as W  # noqa: E402

METRIC = "particle-events/s and s to 1% std-err kappa_eff, batched FP32 vs plain FP64, 1 GB300"
UNIT = "particle-events/s"
WORKLOADS = {"si_slab": "si_slab_L1um_3000bins", "si_slab_imp": "si_slab_L1um_3000bins_two_phonon_clock",
             "transient_box": "transient_box_2x2x1um_gauss",
             "transient_box_avg": "transient_box_2x2x1um_gauss_bin_averages",
             "nanomesh": "nanomesh_W34nm_pore11nm_t22nm_timp",
             "film_batch": "film_batch_64_10nm_10um", "pore_grad": "pore_film_W100nm_phi0.25_t200nm_grad",
             "pore_nscat": "pore_skew_W100nm_phi0.25_t200nm_nscat_curve_1_32"}
# Issue-rate roofline of the FP32 steady tracer: SMs x 4 schedulers x 32
# lanes x f_clk thread-instructions per second, against the instructions one
# event costs, taken from ncu's instruction counters of the bench's own launch
# (smsp__thread_inst_executed.sum and smsp__inst_executed.sum over the tracing
# kernels of one step, divided by the step's events; the capture and its
# command are summarised under profiles/).  Workloads
# without such a capture fall back to the count of the work one event needs
# (one Philox4x32-10 call, log + sqrt + sincos, six-plane first hit, alias
# draw, state update and tallies: 200 thread-instructions).
INSTR_PER_EVENT = 200.0
NCU_INSTR_PER_EVENT = {   # workload: (thread-instructions, warp-instructions) per event
    "si_slab": (375.9, 19.06),    # 2.488e11 / 1.261e10 instructions over 6.619e8 events
}
# DRAM bytes per launch of the FP32 steady tracing kernel on the default
# workload, from the ncu capture summarised in profiles/ (None until a capture
# of the current kernel exists).
TRACE_DRAM_BYTES_PER_LAUNCH = 1_713_152 + 40_448


PROBE_SRC = os.path.join(ROOT, "bench_l2_probe.cu")
PROBE_LIB = os.path.join(ROOT, "bench_l2_probe.so")


def build_probe(force: bool = False) -> str:
    """Compile the bench's L2 reduction probe (bench_l2_probe.cu, not part of
    the library) for sm_103a beside this file."""
    if not force and os.path.exists(PROBE_LIB) and os.path.getmtime(PROBE_LIB) >= os.path.getmtime(PROBE_SRC):
        return PROBE_LIB
    nvcc = "nvcc" if subprocess.run(["which", "nvcc"], capture_output=True).returncode == 0 else "/usr/local/cuda/bin/nvcc"
    subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-shared",
                           "-Xcompiler", "-fPIC", PROBE_SRC, "-o", PROBE_LIB + ".tmp"])
    os.replace(PROBE_LIB + ".tmp", PROBE_LIB)
    return PROBE_LIB


def load_probe():
    build_probe()
    lib = ctypes.CDLL(PROBE_LIB)
    lib.bench_l2_reduction_probe.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p]
    lib.bench_l2_reduction_probe.restype = ctypes.c_int
    return lib


def _dist():
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index: int):
        self.index, self.proc, self.path = index, None, None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(float(r[1]) for r in rows), "sm_max_mhz": float(rows[0][2]),
                "samples": len(rows), "reasons": sorted(reasons)}


def _material_bytes(mat) -> int:
    cols = [mat.omega, mat.v, mat.tau] + ([mat.C] if mat.C is not None else [mat.D, mat.domega])
    return sum(int(c.nbytes) for c in cols)


class Timer:
    """Per-step CUDA events around a step and, recorded by the library on the
    launch stream, around its tracing kernel."""

    def __init__(self):
        import torch
        self.torch = torch
        E = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
        self.s0, self.s1, self.k0, self.k1 = E(), E(), E(), E()
        self.flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")   # > 129 MB L2

    def run(self, step, steps):
        stream = self.torch.cuda.current_stream()
        step_ms, kern_ms, results = [], [], []
        for _ in range(steps):
            self.flush.zero_()                      # L2 flush between timed steps
            # torch only times events it recorded itself: record the kernel
            # events here; the library re-records them on the same stream just
            # before and after the tracing kernel, elapsed_time uses the latest.
            self.k0.record(stream)
            self.k1.record(stream)
            self.s0.record(stream)
            r = step()
            self.s1.record(stream)
            self.s1.synchronize()
            step_ms.append(self.s0.elapsed_time(self.s1))
            kern_ms.append(self.k0.elapsed_time(self.k1))
            results.append(r())
        return step_ms, kern_ms, results


def _tail_kernel(cfg) -> int:
    """1 when the FP32 run hands its last particles to the tail kernel (a
    second launch), else 0."""
    from paper_2104_03573_gb300 import _lib as L
    return int(cfg.precision == L.FP32_TRACE and cfg.tail_lanes >= 0)


def _split(cfg, n_per_geom, rank, world):
    """Steady runs on several GPUs: rank r traces particles [r n, (r+1) n) of
    a run of world x n particles per geometry (weak scaling, per-GPU work
    fixed; the ranks together trace exactly the particles of that run)."""
    if world <= 1:
        return cfg
    return replace(cfg, pid_begin=[rank * int(n) for n in n_per_geom], n_total=[world * int(n) for n in n_per_geom])


def _workload_setup(name, args, seed_offset, rank=0, world=1):
    """Build (material, geometries, step factory, description, counters)."""
    from paper_2104_03573_gb300 import api, _lib as L, batch, autotune
    import torch
    tm = Timer()
    ev = (tm.k0, tm.k1)
    if name in ("si_slab", "si_slab_imp"):
        wl = W.si_slab_c2(n=args.n_particles or 10_000_000)
        mat, geo, run = wl.material, wl.geometries[0], wl.run
        if name == "si_slab_imp":        # separate impurity clock, tau_imp^-1 = 2e-44 omega^4 (s^-1)
            mat = replace(mat, tau_imp=1.0 / (2e-44 * mat.omega ** 4))
        M, G = api.Material(mat), api.Geometry(geo)
        cfg = api.SteadyConfig(seed=run.seed + seed_offset, precision=L.FP32_TRACE, n_cells=run.n_cells,
                               cell_axis=2, tally_axis=2, per_bin=True, threads_per_block=args.threads,
                               blocks_per_sm=args.blocks_per_sm, refill_threshold=args.refill, tail_lanes=args.tail,
                               cell_flux_axis=True)
        if args.threads == 0 and not args.no_autotune:
            # on the whole workload: a smaller sample ranks the shapes by their drain tail
            cfg = autotune.tune(M, [G], [run.n], cfg, fraction=1.0)
        cfg = _split(replace(cfg, trace_events=ev), [run.n], rank, world)
        ws = torch.empty(api.steady_workspace_size(M, [G], [run.n], cfg), dtype=torch.uint8, device="cuda")
        out = api.SteadyOutputs(1, M.n_bins, run.n_cells, True)

        def step():
            api.run_steady(M, [G], [run.n], cfg, out=out, workspace=ws)
            return lambda: out.stats.cpu().numpy()

        def fp64(n64):
            c = replace(cfg, precision=L.FP64_PLAIN, pid_begin=(), n_total=(), threads_per_block=0, refill_threshold=0)
            o = api.SteadyOutputs(1, M.n_bins, run.n_cells, True)
            return lambda: (api.run_steady(M, [G], [n64], c, out=o), (lambda: o.stats.cpu().numpy()))[1]

        def e2e():
            Mh, Gh = api.Material(mat), api.Geometry(geo)
            res = api.run_steady_host(Mh, [Gh], [run.n], replace(cfg, trace_events=None))
            return res["stats"]
        d2h = 8 * (run.n_cells + 3 * run.n_cells + M.n_bins + L.NSTATS)
        h2d = _material_bytes(mat) + ctypes.sizeof(L.GeometryDesc) + 8
        desc = ("steady cross-plane Si-like film L=1um (1um cube, periodic x,y), BvK 3x1000 bins + Holland tau "
                "at 300 K, walls 300+-0.5 K, 50 cells x {T, q_z} + per-bin q_z; FP32 tracing, fixed-point FP64-exact tallies"
                + ("; separate two-phonon clock, tau_imp^-1 = 2e-44 omega^4" if name == "si_slab_imp" else ""))
        launches = 3 + _tail_kernel(cfg)       # setup, tracer (+ tail kernel), finaliser
        shape = {"threads_per_block": cfg.threads_per_block, "refill_threshold": cfg.refill_threshold,
                 "tail_lanes": cfg.tail_lanes}
        return dict(mat=mat, geo=geo, run=run, n=run.n, step=step, fp64=fp64, e2e=e2e, d2h=d2h, h2d=h2d, desc=desc,
                    launches=launches, timer=tm, kernel="k_steady_f32", shape=shape, kappa=True, kind="steady")
    if name == "nanomesh":
        # the paper's nanomesh (Sec. 5.5): N = 1e6, N_scat^max = 10, square pore
        # as four internal walls, diffuse walls, tau_imp^-1 = 2e-44 omega^4
        n = args.n_particles or 1_000_000
        base = W.bvk_holland()
        mat = replace(base, tau_imp=1.0 / (2e-44 * base.omega ** 4))
        geo = W.nanomesh()
        run = W.SteadyRun(n=n, seed=1006 + seed_offset, tally_axis=1, per_bin=True, n_scat_max=10)
        M, G = api.Material(mat), api.Geometry(geo)
        cfg = api.SteadyConfig(seed=run.seed, precision=L.FP32_TRACE, tally_axis=1, per_bin=True, n_scat_max=10,
                               max_events=10 ** 9, threads_per_block=args.threads, refill_threshold=args.refill,
                               time_budget_s=300, tail_lanes=args.tail)
        if args.threads == 0 and not args.no_autotune:
            cfg = autotune.tune(M, [G], [n], cfg)
        cfg = _split(replace(cfg, trace_events=ev), [n], rank, world)
        out = api.SteadyOutputs(1, M.n_bins, 0, True)

        def step():
            api.run_steady(M, [G], [n], cfg, out=out)
            return lambda: out.stats.cpu().numpy()

        def fp64(n64):
            c = replace(cfg, precision=L.FP64_PLAIN, pid_begin=(), n_total=(), threads_per_block=0, refill_threshold=0)
            o = api.SteadyOutputs(1, M.n_bins, 0, True)
            return lambda: (api.run_steady(M, [G], [n64], c, out=o), (lambda: o.stats.cpu().numpy()))[1]

        def e2e():
            Mh, Gh = api.Material(mat), api.Geometry(geo)
            return api.run_steady_host(Mh, [Gh], [n], replace(cfg, trace_events=None))["stats"]
        desc = ("Si nanomesh unit cell 34 nm, 11 nm square pore (four internal walls) through a 22 nm film, "
                "diffuse walls, periodic x,y, grad_T -1e6 K/m along y, BvK 3x1000 bins + Holland tau, "
                "separate impurity clock tau_imp^-1 = 2e-44 omega^4, N_scat_max 10")
        return dict(mat=mat, geo=geo, run=run, n=n, step=step, fp64=fp64, e2e=e2e,
                    d2h=8 * (M.n_bins + L.NSTATS), h2d=_material_bytes(mat) + ctypes.sizeof(L.GeometryDesc) + 8,
                    desc=desc, launches=3 + _tail_kernel(cfg), timer=tm, kernel="k_steady_f32 (nanomesh)",
                    shape={"threads_per_block": cfg.threads_per_block, "refill_threshold": cfg.refill_threshold,
                           "tail_lanes": cfg.tail_lanes},
                    kappa=True, kind="steady")
    if name == "pore_nscat":
        n = args.n_particles or 10_000_000
        mat, geo = W.bvk_holland(), W.pore_skew()
        run = W.SteadyRun(n=n, seed=1007 + seed_offset, tally_axis=1, per_bin=True, n_scat_max=32)
        M, G = api.Material(mat), api.Geometry(geo)
        cfg = api.SteadyConfig(seed=run.seed, precision=L.FP32_TRACE, tally_axis=1, per_bin=True, n_scat_max=32,
                               max_events=10 ** 9, threads_per_block=args.threads, refill_threshold=args.refill,
                               time_budget_s=300, nscat_curve=True, tail_lanes=args.tail)
        if args.threads == 0 and not args.no_autotune:
            cfg = autotune.tune(M, [G], [n], cfg)
        cfg = _split(replace(cfg, trace_events=ev), [n], rank, world)
        out = api.SteadyOutputs(1, M.n_bins, 0, True, nscat=32)

        def step():
            api.run_steady(M, [G], [n], cfg, out=out)
            return lambda: out.stats.cpu().numpy()

        def fp64(n64):
            c = replace(cfg, precision=L.FP64_PLAIN, pid_begin=(), n_total=(), threads_per_block=0, refill_threshold=0)
            o = api.SteadyOutputs(1, M.n_bins, 0, True, nscat=32)
            return lambda: (api.run_steady(M, [G], [n64], c, out=o), (lambda: o.stats.cpu().numpy()))[1]

        def e2e():
            Mh, Gh = api.Material(mat), api.Geometry(geo)
            return api.run_steady_host(Mh, [Gh], [n], replace(cfg, trace_events=None))["stats"]
        desc = ("nanoporous cell without symmetry: 100 nm cell, cylindrical pore porosity 0.25 centred at "
                "(30, 62) nm, 200 nm thick, diffuse walls, periodic x,y, grad_T (-0.5, -1, 0) x 1e6 K/m, "
                "BvK 3x1000 bins + Holland tau; kappa and its SE for every N_scat_max = 1..32 from one run")
        return dict(mat=mat, geo=geo, run=run, n=n, step=step, fp64=fp64, e2e=e2e, curve=out,
                    d2h=8 * (M.n_bins + L.NSTATS + 64), h2d=_material_bytes(mat) + ctypes.sizeof(L.GeometryDesc) + 8,
                    desc=desc, launches=3 + _tail_kernel(cfg), timer=tm, kernel="k_steady_f32 (N_scat_max curve)",
                    shape={"threads_per_block": cfg.threads_per_block, "refill_threshold": cfg.refill_threshold,
                           "tail_lanes": cfg.tail_lanes},
                    kappa=True, kind="steady")
    if name == "pore_grad":
        wl = W.pore_film_c5(n=args.n_particles or 50_000_000)
        mat, geo, run = wl.material, wl.geometries[0], wl.run
        M, G = api.Material(mat), api.Geometry(geo)
        cfg = api.SteadyConfig(seed=run.seed + seed_offset, precision=L.FP32_TRACE, tally_axis=1, per_bin=True,
                               n_scat_max=10, max_events=10 ** 9, threads_per_block=args.threads or 512,
                               refill_threshold=args.refill or 4, trace_events=ev, time_budget_s=300,
                               tail_lanes=args.tail)
        cfg = _split(cfg, [run.n], rank, world)
        fwd = api.SteadyOutputs(1, M.n_bins, 0, True)
        go = api.GradOutputs(M.n_bins)

        def step():
            api.grad(M, G, run.n, cfg, fwd=fwd, gout=go)
            return lambda: fwd.stats.cpu().numpy()

        def fp64(n64):
            c = replace(cfg, precision=L.FP64_PLAIN, pid_begin=(), n_total=())
            f2, g2 = api.SteadyOutputs(1, M.n_bins, 0, True), api.GradOutputs(M.n_bins)
            return lambda: (api.grad(M, G, n64, c, fwd=f2, gout=g2), (lambda: f2.stats.cpu().numpy()))[1]

        def e2e():
            import torch as t
            Mh, Gh = api.Material(mat), api.Geometry(geo)
            f3, g3 = api.grad(Mh, Gh, run.n, replace(cfg, trace_events=None))
            return f3.stats.cpu().numpy(), g3.dkappa_dlogtau.cpu().numpy()
        def nscat_check():
            # N_scat_max convergence check of this workload (the pore lattice's
            # truncation biases kappa): one run with N_scat_max = 40, kappa at 10/20/40
            c = replace(cfg, n_scat_max=40, nscat_curve=True, trace_events=None)
            o = api.run_steady(M, [G], [run.n], c)
            kn = o.kappa_nscat[0].cpu().numpy()
            return {"n_scat_max": [10, 20, 40], "kappa": [float(kn[k - 1, 0]) for k in (10, 20, 40)],
                    "kappa_se": [float(kn[k - 1, 1]) for k in (10, 20, 40)], "particles": int(run.n)}
        desc = ("nanoporous film: 100 nm cell, cylindrical pore porosity 0.25, 200 nm thick, diffuse walls, "
                "grad_T -1e6 K/m along y, N_scat_max 10; forward + gradient: likelihood ratio over 3000 "
                "log-tau scales, measure-valued d kappa / d p_pore at p = 0 (every particle that meets the "
                "pore is traced once more with one pore hit specular)")
        return dict(mat=mat, geo=geo, run=run, n=run.n, step=step, fp64=fp64, e2e=e2e, gout=go, check=nscat_check,
                    d2h=8 * (M.n_bins * 2 + 2 + L.NSTATS), h2d=_material_bytes(mat) + ctypes.sizeof(L.GeometryDesc) + 8,
                    # setup, forward (+ tail), replay (+ tail), finaliser
                    desc=desc, launches=2 + 2 * (1 + _tail_kernel(cfg)), timer=tm, kernel="k_steady_f32 (grad)",
                    shape={"threads_per_block": cfg.threads_per_block, "refill_threshold": cfg.refill_threshold,
                           "tail_lanes": cfg.tail_lanes},
                    kappa=True, kind="grad")
    if name == "film_batch":
        scale = (args.n_particles / 1.4e8) if args.n_particles else 1.0
        wl = W.film_batch_c4(scale=scale)
        mat, run = wl.material, wl.run
        M = api.Material(mat)
        Gs = [api.Geometry(g) for g in wl.geometries]
        cfg = api.SteadyConfig(seed=run.seed + seed_offset, precision=L.FP32_TRACE, tally_axis=1, per_bin=True,
                               n_scat_max=10, max_events=10 ** 9, threads_per_block=args.threads,
                               refill_threshold=args.refill, trace_events=ev, time_budget_s=300,
                               tail_lanes=args.tail)
        cfg = _split(cfg, wl.n_per_geom, rank, world)
        gb = batch.GraphBatch(M, Gs, wl.n_per_geom, cfg, tune=(args.threads == 0 and not args.no_autotune))

        def step():
            gb.replay()
            return lambda: gb.out.stats.cpu().numpy()

        def fp64(n64):
            fr = n64 / sum(wl.n_per_geom)
            ns = [max(1, int(x * fr)) for x in wl.n_per_geom]
            c = replace(cfg, precision=L.FP64_PLAIN, pid_begin=(), n_total=(), trace_events=ev)
            o = api.SteadyOutputs(len(Gs), M.n_bins, 0, True)
            return lambda: (api.run_steady(M, Gs, ns, c, out=o), (lambda: o.stats.cpu().numpy()))[1]

        e2e_k = [0]

        def e2e():
            # the graph replays take keys seed+1, seed+2, ...: end-to-end run k takes
            # the key of timed step k (run 0 is untimed), so both see the same samples
            Mh = api.Material(mat)
            Gh = [api.Geometry(g) for g in wl.geometries]
            key = gb.cfg.seed + args.warmup + e2e_k[0]
            e2e_k[0] += 1
            res = api.run_steady_host(Mh, Gh, wl.n_per_geom, replace(gb.cfg, seed=key, trace_events=None,
                                                                        seed_device=None))
            return res["stats"]
        desc = ("64 in-plane films d = 10 nm * 1000^(f/63), 100x100 nm cell, periodic x,y, diffuse z, grad_T -1e6 K/m, "
                "N_f = 1e5*100^u_f, N_scat_max 10; one persistent launch replayed as a CUDA graph")
        return dict(mat=mat, geo=None, run=run, n=int(sum(wl.n_per_geom)), step=step, fp64=fp64, e2e=e2e,
                    d2h=8 * 64 * (M.n_bins + L.NSTATS),
                    h2d=_material_bytes(mat) + 64 * (ctypes.sizeof(L.GeometryDesc) + 8), desc=desc,
                    launches=3 + _tail_kernel(gb.cfg),
                    timer=tm, kernel="k_steady_f32 (64 geometries, graph)",
                    shape={"threads_per_block": gb.cfg.threads_per_block, "refill_threshold": gb.cfg.refill_threshold,
                           "tail_lanes": gb.cfg.tail_lanes},
                    kappa=True, kind="batch")
    if name in ("transient_box", "transient_box_avg"):
        wl = W.transient_box_c3(n=args.n_particles or 100_000_000)
        mat, geo, run = wl.material, wl.geometries[0], wl.run
        run.time_average = name == "transient_box_avg"
        M, G = api.Material(mat), api.Geometry(geo)
        cfg = api.TransientConfig(seed=run.seed + seed_offset, t_max=run.t_max, t_meas=run.t_meas, grid=run.grid,
                                  precision=L.FP32_TRACE, threads_per_block=args.threads if args.threads in (0, 256, 512, 768, 1024) else 0,
                                  trace_events=ev, time_budget_s=300, time_average=run.time_average)
        out = api.TransientOutputs(len(run.t_meas), run.grid, run.n)

        def step():
            api.run_transient(M, G, run.n, cfg, out=out)
            return lambda: out.stats.cpu().numpy()[None, :]

        def fp64(n64):
            c = replace(cfg, precision=L.FP64_PLAIN)
            o = api.TransientOutputs(len(run.t_meas), run.grid, n64)
            return lambda: (api.run_transient(M, G, n64, c, out=o), (lambda: o.stats.cpu().numpy()[None, :]))[1]

        host = {}

        def e2e():
            import numpy as np
            from paper_2104_03573_gb300 import _lib as LL
            Mh, Gh = api.Material(mat), api.Geometry(geo)
            nx, ny, nz = run.grid
            if not host:
                # the result's host buffers, pinned, allocated once (the first,
                # untimed call): each step reads its 839 MB tally into them
                host["tally"] = torch.zeros((len(run.t_meas), nz, ny, nx, 4), dtype=torch.float64).pin_memory().numpy()
                host["st"] = torch.zeros(LL.NSTATS, dtype=torch.float64).pin_memory().numpy()
            tally, st = host["tally"], host["st"]
            tmv = np.ascontiguousarray(run.t_meas, dtype=np.float64)
            p = api.transient_params(replace(cfg, trace_events=None), run.n, tmv)
            o = LL.TransientOut()
            o.tally, o.stats, o.on_host = tally.ctypes.data, st.ctypes.data, 1
            LL.check(LL.load().mcbte_run_transient(Mh.handle, Gh.handle, ctypes.byref(p), ctypes.byref(o), None, 0,
                                                   None), allow=(LL.OK, LL.WARN_TRUNCATED))
            return st[None, :]
        nt = len(run.t_meas) * run.grid[0] * run.grid[1] * run.grid[2] * 4 * 8
        # time windows of the FP32 run (the library's automatic choice: the
        # largest window whose tally slice fits a third of the L2)
        slice_b = run.grid[0] * run.grid[1] * run.grid[2] * 4 * 8
        l2 = int(getattr(torch.cuda.get_device_properties(torch.cuda.current_device()), "L2_cache_size", 96 << 20))
        wt = max(1, min(len(run.t_meas), (l2 // 3) // slice_b))
        windows = -(-len(run.t_meas) // wt)
        desc = ("transient 2x2x1 um diffuse adiabatic box, +1 K Gaussian sigma 100 nm at the top-face centre, "
                "64x64x32 cells x 200 " + ("10 ps bin averages" if run.time_average else "snapshots (10 ps)")
                + ", FP32 flights, fixed-point tallies in L2-sized time windows")
        return dict(mat=mat, geo=geo, run=run, n=run.n, step=step, fp64=fp64, e2e=e2e, d2h=nt + 8 * L.NSTATS,
                    h2d=_material_bytes(mat) + ctypes.sizeof(L.GeometryDesc) + 8 * len(run.t_meas), desc=desc,
                    launches=2 + windows, timer=tm, kernel="k_transient_f32",
                    shape={"threads_per_block": cfg.threads_per_block, "time_windows": windows},
                    kappa=False, kind="transient",
                    # adiabatic box: every particle lives to t_max, so it is sampled at all n_times
                    tally_ops=run.n * len(run.t_meas), l2_slice_words=wt * slice_b // 8)
    raise ValueError(name)


def run_ours(args):
    import numpy as np
    import torch

    ws, rank, lrank = _dist()
    torch.cuda.set_device(lrank)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", lrank))
    from paper_2104_03573_gb300 import build, _lib as L
    build.build()
    from paper_2104_03573_gb300 import shard
    # steady workloads: rank r traces its own range of a world x n particle run
    # under the one key; the transient box (no range split) takes a key per rank
    wk = _workload_setup(args.workload, args, shard.rank_key(0, rank) if args.workload.startswith("transient") else 0,
                         rank, ws)
    tm = wk["timer"]
    for _ in range(args.warmup):
        wk["step"]()()
    torch.cuda.synchronize()
    sampler = ClockSampler(lrank)
    sampler.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    step_ms, kern_ms, stats = tm.run(wk["step"], args.steps)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    wall = time.perf_counter() - t0
    clocks = sampler.stop()
    for st in stats:
        assert np.all(st[:, L.STAT_STATUS] == 0), f"run status {st[:, L.STAT_STATUS]}"
    t_step = sum(step_ms) / len(step_ms) / 1e3
    ev_step = float(np.mean([st[:, L.STAT_EVENTS].sum() for st in stats]))
    total_events, t_ranks, wall_max = ev_step * args.steps, t_step * args.steps, wall
    if dist:
        # weak scaling: every rank's events count, the slowest rank sets the time
        total_events = shard.sum_over_ranks(total_events)
        t_ranks = shard.max_over_ranks(t_ranks)
        wall_max = shard.max_over_ranks(wall_max)
    value = total_events / t_ranks
    st = stats[-1]
    kappa = kse = t_1pct = None
    if wk["kappa"]:
        k = st[:, L.STAT_KAPPA]
        se = st[:, L.STAT_KAPPA_SE]
        kappa, kse = float(k[0]), float(se[0])
        if dist:                                        # pooled over the ranks' independent samples
            pooled = shard.pooled_kappa(shard.allreduce_stats(st)[0])
            kappa, kse = pooled["kappa"], pooled["kappa_se"]
        t_1pct = float(t_step * np.max((se / np.abs(k) / 0.01) ** 2))
    dkdp = [float(x) for x in wk["gout"].dkappa_dp.cpu().numpy()] if "gout" in wk else None
    curve = None
    check = wk["check"]() if "check" in wk else None
    l2 = l2_reduction_roofline(wk, t_kern_probe(kern_ms)) if "tally_ops" in wk else None
    if "curve" in wk:
        kn = wk["curve"].kappa_nscat[0].cpu().numpy()
        kfin, sfin = kn[-1]
        # the smallest N_scat_max whose kappa is within two standard errors of the largest one's
        conv = next(k + 1 for k in range(len(kn)) if abs(kn[k, 0] - kfin) <= 2.0 * np.hypot(kn[k, 1], sfin))
        curve = {"n_scat_max": [1, 2, 4, 8, 16, 32], "kappa": [float(kn[k - 1, 0]) for k in (1, 2, 4, 8, 16, 32)],
                 "kappa_se": [float(kn[k - 1, 1]) for k in (1, 2, 4, 8, 16, 32)], "converged_at": int(conv)}
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    fp64 = None
    if not args.no_fp64:
        n64 = args.fp64_particles or (10_000_000 if args.workload == "si_slab" else 2_000_000)
        f = wk["fp64"](n64)
        f()()                                           # warm-up
        torch.cuda.synchronize()
        s_ms, _, st64 = tm.run(f, 1)
        t64 = s_ms[0] / 1e3
        s64 = st64[0]
        fp64 = {"value": float(s64[:, L.STAT_EVENTS].sum() / t64), "unit": UNIT, "n_particles": n64, "s_per_run": t64}
        if wk["kappa"]:
            se64 = s64[:, L.STAT_KAPPA_SE] / np.abs(s64[:, L.STAT_KAPPA])
            fp64.update({"kappa": float(s64[0, L.STAT_KAPPA]), "kappa_se": float(s64[0, L.STAT_KAPPA_SE]),
                         "s_to_1pct_se": float(t64 * np.max((se64 / 0.01) ** 2))})

    # end-to-end through the public API with host buffers: material upload and
    # table build, geometry upload, run with host outputs (copies back and
    # synchronises), release
    e2e_times, n_e2e = [], max(1, min(args.steps, 3))
    ev_e2e = None
    for k in range(n_e2e + 1):
        torch.cuda.synchronize()
        t_a = time.perf_counter()
        r = wk["e2e"]()
        t_b = time.perf_counter()
        if k > 0:
            e2e_times.append(t_b - t_a)
        ev_e2e = float(np.asarray(r[0] if isinstance(r, tuple) else r)[:, L.STAT_EVENTS].sum())
    t_e2e = sum(e2e_times) / len(e2e_times)

    peaks, peak_kind = _peaks()
    n_sm = torch.cuda.get_device_properties(lrank).multi_processor_count
    f_max = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    peak_tinst = n_sm * 4 * 32 * f_max / 1e12
    t_kern = sum(kern_ms) / len(kern_ms) / 1e3
    roof = _roofline(args.workload, ev_step, t_kern, n_sm, f_max, peak_kind)
    roof.update({"traffic": TRACE_DRAM_BYTES_PER_LAUNCH if args.workload == "si_slab" else None,
                 "kernel": wk["kernel"], "kernel_ms": t_kern * 1e3})
    subs = _sub_records(args, lrank) if (ws == 1 and args.workload == "si_slab" and args.sub_steps > 0) else None
    cpu = cpu_baseline(wk, args) if (ws == 1 and not args.no_cpu) else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "description": wk["desc"], "n_particles_per_gpu": wk["n"],
                   "parallelism": f"independent samples x{ws}",
                   "l2": "256 MiB buffer zeroed between timed steps (outside the per-step CUDA events)",
                   "seed": wk["run"].seed, "launch": wk["shape"]},
        "s_to_1pct_se_kappa": t_1pct, "kappa_eff": kappa, "kappa_se": kse,
        "events_per_step": ev_step, "wall_s": wall_max,
        **({"dkappa_dp_pore": dkdp} if dkdp is not None else {}),
        **({"kappa_nscat": curve} if curve is not None else {}),
        **({"nscat_check": check} if check is not None else {}),
        **({"l2_reductions": l2} if l2 is not None else {}),
        **({"tally_ops_per_s": {"value": wk["tally_ops"] * args.steps * ws / t_ranks,
                                "what": "snapshot tallies (4 atomics each) per second"}}
           if "tally_ops" in wk else {}),
        "fp64_plain": fp64,
        "roofline": roof,
        **({"workloads": subs} if subs else {}),
        "e2e": {"value": ev_e2e / t_e2e, "unit": UNIT, "h2d_bytes_per_step": int(wk["h2d"]),
                "d2h_bytes_per_step": int(wk["d2h"]), "s_per_step": t_e2e},
        "gpu_launches": wk["launches"] * args.steps,
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def _roofline(workload, ev_step, t_kern, n_sm, f_max, peak_kind):
    """Issue-rate roofline of the tracing kernels of one step: achieved
    thread-instructions per second (events x instructions per event / kernel
    time) against SMs x 4 x 32 x f_max; issue_frac is the same with warp
    instructions against SMs x 4 x f_max, simt_eff the mean active lanes per
    warp instruction over 32."""
    peak = n_sm * 4 * 32 * f_max / 1e12
    if workload in NCU_INSTR_PER_EVENT:
        ti, wi = NCU_INSTR_PER_EVENT[workload]
        achieved = ev_step * ti / t_kern / 1e12
        return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tinst/s", "frac": achieved / peak,
                "issue_frac": ev_step * wi / t_kern / (n_sm * 4 * f_max), "simt_eff": ti / (32.0 * wi),
                "thread_inst_per_event": ti, "warp_inst_per_event": wi,
                "frac_200_algorithmic": ev_step * INSTR_PER_EVENT / t_kern / 1e12 / peak,
                "peak_basis": f"{n_sm} SMs x 4 x 32 lanes x {f_max / 1e6:.0f} MHz ({peak_kind} sm_max_mhz); "
                              f"{ti:.1f} thread- / {wi:.2f} warp-instructions per event from ncu instruction "
                              f"counters of this launch"}
    achieved = ev_step * INSTR_PER_EVENT / t_kern / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tinst/s", "frac": achieved / peak,
            "peak_basis": f"{n_sm} SMs x 4 x 32 lanes x {f_max / 1e6:.0f} MHz ({peak_kind} sm_max_mhz); "
                          f"{INSTR_PER_EVENT:.0f} thread-instructions per event (work count; no ncu count of "
                          f"this workload)"}


def _sub_records(args, dev):
    """The default run's extra lines: the film batch under a CUDA graph, the
    transient box and the pore-film gradient, each W = 3 warm-up and
    args.sub_steps timed steps (L2 flushed between steps, CUDA events, clocks
    sampled), in the same units as the main line."""
    import numpy as np
    import torch
    from paper_2104_03573_gb300 import _lib as L
    out = {}
    for name in ("film_batch", "transient_box", "pore_grad"):
        sa = argparse.Namespace(**vars(args))
        sa.n_particles, sa.threads, sa.blocks_per_sm, sa.refill, sa.workload = 0, 0, 0, 0, name
        wk = _workload_setup(name, sa, 0)
        tm = wk["timer"]
        for _ in range(3):
            wk["step"]()()
        torch.cuda.synchronize()
        sampler = ClockSampler(dev)
        sampler.start()
        step_ms, kern_ms, stats = tm.run(wk["step"], args.sub_steps)
        torch.cuda.synchronize()
        clocks = sampler.stop()
        for st in stats:
            assert np.all(st[:, L.STAT_STATUS] == 0), f"{name}: run status {st[:, L.STAT_STATUS]}"
        t_step = sum(step_ms) / len(step_ms) / 1e3
        t_kern = sum(kern_ms) / len(kern_ms) / 1e3
        ev = float(np.mean([st[:, L.STAT_EVENTS].sum() for st in stats]))
        rec = {"workload": WORKLOADS[name], "description": wk["desc"], "value": ev / t_step, "unit": UNIT,
               "ms_per_step": t_step * 1e3, "kernel_ms": t_kern * 1e3, "steps": args.sub_steps, "warmup": 3,
               "events_per_step": ev, "n_particles": wk["n"], "launch": wk["shape"],
               "ms_per_step_each": [round(x, 3) for x in step_ms], "clocks": clocks}
        st = stats[-1]
        if wk["kappa"]:
            k, se = st[:, L.STAT_KAPPA], st[:, L.STAT_KAPPA_SE]
            rec["s_to_1pct_se_kappa"] = float(t_step * np.max((se / np.abs(k) / 0.01) ** 2))
            rec["kappa_eff"] = float(k[0]) if k.size == 1 else [round(float(x), 4) for x in k]
        if "gout" in wk:
            rec["dkappa_dp_pore"] = [float(x) for x in wk["gout"].dkappa_dp.cpu().numpy()]
        if "tally_ops" in wk:
            rec["l2_reductions"] = l2_reduction_roofline(wk, t_kern)
            rec["tally_ops_per_s"] = wk["tally_ops"] / t_step
        out[name] = rec
        del wk
        torch.cuda.empty_cache()
    return out


def t_kern_probe(kern_ms):
    return sum(kern_ms) / len(kern_ms) / 1e3


def l2_reduction_roofline(wk, t_kern):
    """Snapshot-bound transient runs: the 64-bit L2 reductions the tracing
    kernels issue per second (4 per snapshot) against the rate the bench's
    probe (bench_l2_probe.cu) reaches in the same pattern on an array the size of one time
    window's tally slice (best of 3 timed launches)."""
    import torch
    from paper_2104_03573_gb300 import _lib as L
    words = int(wk["l2_slice_words"]) // 4 * 4
    slots = torch.zeros(words, dtype=torch.int64, device="cuda")
    groups = 1 << 28
    lib = load_probe()
    s = torch.cuda.current_stream()
    assert lib.bench_l2_reduction_probe(slots.data_ptr(), words, groups // 16, ctypes.c_void_p(s.cuda_stream)) == 0
    best = None
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        assert lib.bench_l2_reduction_probe(slots.data_ptr(), words, groups, ctypes.c_void_p(s.cuda_stream)) == 0
        e1.record(s)
        e1.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        best = t if best is None else min(best, t)
    peak = 4.0 * groups / best / 1e9
    achieved = 4.0 * wk["tally_ops"] / t_kern / 1e9
    return {"achieved": achieved, "peak": peak, "unit": "G reductions/s", "frac": achieved / peak,
            "peak_basis": f"bench_l2_probe.cu: 2^28 groups of 4 64-bit reductions into a "
                          f"{words * 8 / 2**20:.0f} MiB array (one time window's tally slice), best of 3"}


def cpu_baseline(wk, args, target_s=None):
    """The oracle, as it stands, on the host cores: a bounded sample of the
    same workload sized to about `target_s` seconds of CPU work."""
    import oracle
    target_s = target_s or args.cpu_seconds
    run, mat = wk["run"], wk["mat"]
    kind = wk["kind"]
    if kind == "transient":
        def go(n):
            r = W.TransientRun(n=n, seed=run.seed, t_max=run.t_max, t_meas=run.t_meas, grid=run.grid,
                               time_average=bool(getattr(run, "time_average", False)))
            return oracle.run_transient(mat, wk["geo"], r, n_threads=4)
        probe_n = 5_000
        cores = 4
    elif kind == "batch":
        wl = W.film_batch_c4()
        geos = wl.geometries

        def go(n):
            tot_ev, res = 0.0, None
            per = max(1, n // 8)
            for f in range(0, 64, 8):
                r = oracle.run_steady(mat, geos[f], replace(run, max_events=10 ** 9), n_total=per, batch_index=f)
                tot_ev += r["events"]
                res = r
            res = dict(res)
            res["events"] = tot_ev
            return res
        probe_n = 8_000
        cores = os.cpu_count()
    else:
        def go(n):
            r = replace(run, n=n)
            return oracle.run_steady(mat, wk["geo"], r, grad=(kind == "grad"), nscat_curve="curve" in wk)
        probe_n = 50_000
        cores = os.cpu_count()
    t0 = time.perf_counter()
    r0 = go(probe_n)
    dt0 = time.perf_counter() - t0
    n = int(min(wk["n"], max(probe_n, probe_n * target_s / max(dt0, 1e-3))))
    t0 = time.perf_counter()
    r = go(n)
    dt = time.perf_counter() - t0
    out = {"value": r["events"] / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{n} of {wk['n']} particles of the same workload ({r['events']:.3g} events, {dt:.1f} s)"}
    if "kappa" in r and wk["kappa"] and kind != "batch":
        out["s_to_1pct_se_kappa"] = dt * (r["kappa_se"] / abs(r["kappa"]) / 0.01) ** 2
        out["kappa_eff"] = r["kappa"]
    return out


def run_reference(args):
    ws, rank, lrank = _dist()
    if rank != 0:
        return
    mat = W.bvk_holland()
    wl = W.si_slab_c2(n=args.n_particles or 10_000_000, material=mat)
    wk = {"run": wl.run, "mat": mat, "geo": wl.geometries[0], "kind": "steady", "n": wl.run.n, "kappa": True}
    per = max(2.0, min(args.cpu_seconds, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        cpu_baseline(wk, args, target_s=per)
    res = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        res.append(cpu_baseline(wk, args, target_s=per))
    wall = time.perf_counter() - t0
    value = statistics.mean(r["value"] for r in res)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": wall / args.steps * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": WORKLOADS["si_slab"], "n_particles_per_gpu": wl.run.n, "seed": wl.run.seed},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                         "sample": res[-1]["sample"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="si_slab", choices=sorted(WORKLOADS))
    ap.add_argument("--n-particles", type=int, default=0)
    ap.add_argument("--fp64-particles", type=int, default=0)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--blocks-per-sm", type=int, default=0)
    ap.add_argument("--refill", type=int, default=0)
    ap.add_argument("--tail", type=int, default=0,
                    help="tail_lanes of the FP32 steady runs: 0 default / autotuned, -1 no tail kernel")
    ap.add_argument("--sub-steps", type=int, default=3,
                    help="timed steps of each extra workload line of the default run (0: none)")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
