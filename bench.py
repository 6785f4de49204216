#!/usr/bin/env python3
"""Benchmark of the deviational Monte Carlo phonon-BTE hot path on GB300.

Workload (default): steady cross-plane silicon-like film, L = 1 um, BvK
dispersion with 3 x 1000 bins and Holland relaxation times at 300 K, walls at
300 +/- 0.5 K, 1e7 deviational particles, 50 track-length cells and the
frequency-resolved flux (3000 bins).  One step = one full run of the hot
path: run setup, tracing of all 1e7 particles, finalisation.

Our arm times the persistent FP32 tracer (FP64 tallies) and reports
particle-events/s plus seconds to a 1 % standard error on kappa_eff
(t_run * (SE_rel / 0.01)^2), with the plain FP64 tracer timed beside it on
the same inputs.  ``--impl reference`` times the FP64 CPU oracle on the host
cores on a bounded sample of the same workload.

Multi-GPU (torchrun): every rank traces its own independent 1e7-particle
sample (seed offset by rank): weak scaling, no collective on the data path.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from inputs import workloads as W  # noqa: E402

METRIC = "particle-events/s and s to 1% std-err kappa_eff, batched FP32 vs plain FP64, 1 GB300"
UNIT = "particle-events/s"
WORKLOAD = "si_slab_L1um_3000bins"
# Algorithmic thread-instructions per event of the tracer (one Philox4x32-10
# call, log + sqrt + sincos, six-plane first hit, alias draw, state update and
# tallies); the issue-rate roofline is SMs x 4 x 32 lanes x f_clk / this.
INSTR_PER_EVENT = 200.0
# DRAM bytes per launch of the FP32 tracing kernel on this workload, from the
# ncu capture summarised in profiles/ (None until a capture of the current
# kernel exists).
TRACE_DRAM_BYTES_PER_LAUNCH = None


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    lrank = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, lrank


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
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
        sm = [float(r[1]) for r in rows]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]), "samples": len(rows),
                "reasons": sorted(reasons)}


def _material_bytes(mat) -> int:
    cols = [mat.omega, mat.v, mat.tau] + ([mat.C] if mat.C is not None else [mat.D, mat.domega])
    return sum(int(c.nbytes) for c in cols)


def run_ours(args):
    import numpy as np
    import torch

    ws, rank, lrank = _dist()
    torch.cuda.set_device(lrank)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", lrank))
    from paper_2104_03573_gb300 import build, api, _lib as L
    build.build()
    wl = W.si_slab_c2(n=args.n_particles)
    mat, geo, run = wl.material, wl.geometries[0], wl.run
    M = api.Material(mat)
    G = api.Geometry(geo)
    seed = run.seed + 1_000_003 * rank
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kv0, kv1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    cfg = api.SteadyConfig(seed=seed, precision=L.FP32_TRACE, n_cells=run.n_cells, cell_axis=2, tally_axis=2,
                           per_bin=True, threads_per_block=args.threads, blocks_per_sm=args.blocks_per_sm,
                           refill_threshold=args.refill, trace_events=(kv0, kv1))
    if args.threads == 0 and not args.no_autotune:
        from paper_2104_03573_gb300 import autotune
        from dataclasses import replace
        cfg = replace(autotune.tune(M, [G], [run.n], replace(cfg, trace_events=None)), trace_events=(kv0, kv1))
    launch_shape = {"threads_per_block": cfg.threads_per_block, "blocks_per_sm": cfg.blocks_per_sm,
                    "refill_threshold": cfg.refill_threshold}
    ws_bytes = api.steady_workspace_size(M, [G], [run.n], cfg)
    workspace = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    out = api.SteadyOutputs(1, M.n_bins, run.n_cells, True)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")   # > 129 MB L2
    stream = torch.cuda.current_stream()

    def step():
        api.run_steady(M, [G], [run.n], cfg, out=out, workspace=workspace, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(lrank)
    sampler.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms, kern_ms, events, kappas, kses = [], [], [], [], []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()                                   # L2 flush between timed steps
        # torch only times events it has recorded itself: record the kernel
        # events once here; the library re-records them on the same stream
        # just before and after the tracing kernel, and elapsed_time uses the
        # latest records.
        kv0.record(stream)
        kv1.record(stream)
        ev0.record(stream)
        step()
        ev1.record(stream)
        ev1.synchronize()
        step_ms.append(ev0.elapsed_time(ev1))
        kern_ms.append(kv0.elapsed_time(kv1))
        st = out.stats[0].cpu().numpy()
        events.append(st[L.STAT_EVENTS])
        kappas.append(st[L.STAT_KAPPA])
        kses.append(st[L.STAT_KAPPA_SE])
        assert st[L.STAT_STATUS] == 0, f"run status {st[L.STAT_STATUS]}"
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    wall = time.perf_counter() - t0
    clocks = sampler.stop()

    t_step = sum(step_ms) / len(step_ms) / 1e3            # s, device time of one step on this rank
    ev_step = float(np.mean(events))
    tot = torch.tensor([ev_step * args.steps, t_step * args.steps, wall], dtype=torch.float64, device="cuda")
    if dist:
        s = tot.clone()
        dist.all_reduce(s[0:1], op=dist.ReduceOp.SUM)
        dist.all_reduce(s[1:3], op=dist.ReduceOp.MAX)
        tot = s
    total_events, t_max_ranks, wall_max = (float(x) for x in tot.cpu())
    value = total_events / t_max_ranks
    kappa = float(np.mean(kappas))
    se_rel = float(np.mean(kses)) / kappa
    t_1pct = t_step * (se_rel / 0.01) ** 2

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    # plain FP64 tracer on the same inputs (one timed run after one warm-up)
    fp64 = None
    if not args.no_fp64:
        c64 = api.SteadyConfig(seed=seed, precision=L.FP64_PLAIN, n_cells=run.n_cells, cell_axis=2, tally_axis=2,
                               per_bin=True, trace_events=(kv0, kv1))
        o64 = api.SteadyOutputs(1, M.n_bins, run.n_cells, True)
        n64 = args.fp64_particles
        api.run_steady(M, [G], [n64], c64, out=o64)
        torch.cuda.synchronize()
        flush.zero_()
        kv0.record(stream)
        kv1.record(stream)
        ev0.record(stream)
        api.run_steady(M, [G], [n64], c64, out=o64, stream=stream)
        ev1.record(stream)
        ev1.synchronize()
        t64 = ev0.elapsed_time(ev1) / 1e3
        s64 = o64.stats[0].cpu().numpy()
        se64 = s64[L.STAT_KAPPA_SE] / s64[L.STAT_KAPPA]
        fp64 = {"value": s64[L.STAT_EVENTS] / t64, "unit": UNIT, "n_particles": n64, "s_per_run": t64,
                "kappa": s64[L.STAT_KAPPA], "kappa_se": s64[L.STAT_KAPPA_SE],
                "s_to_1pct_se": t64 * (se64 / 0.01) ** 2}

    # end-to-end through the public API with host buffers: material upload and
    # table build, run with host outputs (copies back, synchronises), release
    e2e_times = []
    n_e2e = max(1, min(args.steps, 3))
    for k in range(n_e2e + 1):
        t_a = time.perf_counter()
        Mh = api.Material(mat)
        Gh = api.Geometry(geo)
        res = api.run_steady_host(Mh, [Gh], [run.n], cfg_host(api, L, run, seed))
        del Mh, Gh
        t_b = time.perf_counter()
        if k > 0:
            e2e_times.append(t_b - t_a)
        ev_e2e = res["stats"][0][L.STAT_EVENTS]
    t_e2e = sum(e2e_times) / len(e2e_times)
    import ctypes
    # material columns + geometry descriptor + the n_particles word
    h2d = _material_bytes(mat) + ctypes.sizeof(L.GeometryDesc) + 8
    d2h = 8 * (run.n_cells + 3 * run.n_cells + M.n_bins + L.NSTATS)

    peaks, peak_kind = _peaks()
    props = torch.cuda.get_device_properties(lrank)
    n_sm = props.multi_processor_count
    f_max = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    peak_tinst = n_sm * 4 * 32 * f_max / 1e12
    t_kern = sum(kern_ms) / len(kern_ms) / 1e3
    achieved = ev_step * INSTR_PER_EVENT / t_kern / 1e12

    cpu = cpu_baseline(mat, geo, run, args) if (ws == 1 and not args.no_cpu) else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "description": "steady cross-plane Si-like film L=1um, BvK 3x1000 bins + "
                   "Holland tau at 300 K, walls 300+-0.5 K, 50 cells + per-bin flux; FP32 tracing, FP64 tallies",
                   "n_particles_per_gpu": run.n, "parallelism": f"independent samples x{ws}",
                   "l2": "256 MiB buffer zeroed between timed steps (outside the per-step CUDA events)",
                   "seed": run.seed, "launch": launch_shape},
        "s_to_1pct_se_kappa": t_1pct, "kappa_eff": kappa, "kappa_se": float(np.mean(kses)),
        "events_per_step": ev_step, "wall_s": wall_max,
        "fp64_plain": fp64,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tinst, "unit": "Tinst/s",
                     "frac": achieved / peak_tinst, "traffic": TRACE_DRAM_BYTES_PER_LAUNCH,
                     "kernel": "k_steady_f32", "kernel_ms": t_kern * 1e3,
                     "peak_basis": f"{n_sm} SMs x 4 x 32 lanes x {f_max / 1e6:.0f} MHz ({peak_kind} sm_max_mhz); "
                                   f"{INSTR_PER_EVENT:.0f} algorithmic thread-instructions per event"},
        "e2e": {"value": ev_e2e / t_e2e, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "s_per_step": t_e2e},
        "gpu_launches": 3 * args.steps,
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def cfg_host(api, L, run, seed):
    return api.SteadyConfig(seed=seed, precision=L.FP32_TRACE, n_cells=run.n_cells, cell_axis=2, tally_axis=2,
                            per_bin=True)


def cpu_baseline(mat, geo, run, args, target_s: float = None):
    """The oracle, as it stands, on the host cores: a bounded sample of the
    same workload sized to about `target_s` seconds of CPU work."""
    import oracle
    target_s = target_s or args.cpu_seconds
    probe = W.SteadyRun(n=100_000, seed=run.seed, n_cells=run.n_cells, cell_axis=2, tally_axis=2, per_bin=True)
    t0 = time.perf_counter()
    r0 = oracle.run_steady(mat, geo, probe)
    dt0 = time.perf_counter() - t0
    rate = r0["events"] / dt0
    ev_per_p = r0["events"] / probe.n
    n = int(min(run.n, max(100_000, target_s * rate / ev_per_p)))
    sample = W.SteadyRun(n=n, seed=run.seed, n_cells=run.n_cells, cell_axis=2, tally_axis=2, per_bin=True)
    t0 = time.perf_counter()
    r = oracle.run_steady(mat, geo, sample)
    dt = time.perf_counter() - t0
    se_rel = r["kappa_se"] / r["kappa"]
    return {"value": r["events"] / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{n} of {run.n} particles of the same workload ({r['events']:.3g} events, {dt:.1f} s)",
            "s_to_1pct_se_kappa": dt * (se_rel / 0.01) ** 2, "kappa_eff": r["kappa"]}


def run_reference(args):
    ws, rank, lrank = _dist()
    if rank != 0:
        return
    mat = W.bvk_holland()
    wl = W.si_slab_c2(n=args.n_particles, material=mat)
    geo, run = wl.geometries[0], wl.run
    import oracle
    per = max(2.0, min(args.cpu_seconds, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        cpu_baseline(mat, geo, run, args, target_s=per)
    res = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        res.append(cpu_baseline(mat, geo, run, args, target_s=per))
    wall = time.perf_counter() - t0
    value = statistics.mean(r["value"] for r in res)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": wall / args.steps * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": WORKLOAD, "n_particles_per_gpu": run.n, "seed": run.seed},
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
    ap.add_argument("--n-particles", type=int, default=10_000_000)
    ap.add_argument("--fp64-particles", type=int, default=10_000_000)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--blocks-per-sm", type=int, default=0)
    ap.add_argument("--refill", type=int, default=0)
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
