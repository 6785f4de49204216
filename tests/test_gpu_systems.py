"""Batching, CUDA-graph replay, autotuning and the autograd adjoint.

* launch-shape independence: every particle's random stream is keyed by its
  own id, and the FP32 path accumulates its tallies in 64-bit fixed point,
  so per-particle results and all tallies are bit-identical for every block
  size and refill threshold;
* a captured CUDA graph of a batched multi-geometry run reproduces a direct
  run with the same key, and a new key gives a new sample;
* the torch.autograd.Function backward equals ``mcbte_grad`` and agrees with
  central finite differences under common random numbers.
"""
import math
import ctypes
from dataclasses import replace

import numpy as np
import pytest

from inputs import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2104_03573_gb300 import _lib as L  # noqa: E402
from paper_2104_03573_gb300 import api, autograd, autotune, batch  # noqa: E402
from oracle import closed_forms as cf  # noqa: E402
import oracle  # noqa: E402


def _run(M, Gs, ns, cfg, per_particle=False):
    out = api.run_steady(M, Gs, ns, cfg, per_particle=per_particle)
    torch.cuda.synchronize()
    return out


def test_fp32_results_independent_of_launch_shape():
    wl = W.si_slab_c2(n=60_000)
    mat, geo, run = wl.material, wl.geometries[0], wl.run
    M, G = api.Material(mat), api.Geometry(geo)
    base = None
    for threads, refill in ((256, 1), (512, 1), (768, 8), (1024, 32)):
        cfg = api.SteadyConfig(seed=run.seed, precision=L.FP32_TRACE, n_cells=run.n_cells, tally_axis=2,
                               per_bin=True, threads_per_block=threads, refill_threshold=refill)
        o = _run(M, [G], [run.n], cfg, per_particle=True)
        cur = {k: getattr(o, k).cpu().numpy() for k in ("events_pp", "X_pp", "T", "q", "q_bin")}
        if base is None:
            base = cur
            continue
        for k in cur:
            assert np.array_equal(cur[k], base[k]), (threads, refill, k)


@pytest.mark.parametrize("precision", [L.FP64_PLAIN, L.FP32_TRACE])
def test_run_split_by_particle_ranges_equals_the_whole_run(precision):
    """pid_begin / n_total: three calls that cover a run's particle indices
    trace exactly its particles (per-particle results bit for bit), their
    tallies add up to the run's, and the pooled statistics (shard.combine_stats)
    give the run's kappa and standard error."""
    from paper_2104_03573_gb300 import shard
    wl = W.si_slab_c2(n=90_001)
    mat, geo, run = wl.material, wl.geometries[0], wl.run
    M, G = api.Material(mat), api.Geometry(geo)
    cfg = api.SteadyConfig(seed=run.seed, precision=precision, n_cells=run.n_cells, cell_axis=2, tally_axis=2,
                           per_bin=True)
    full = _run(M, [G], [run.n], cfg, per_particle=True)
    parts = []
    for r in range(3):
        c, ns = shard.rank_config(cfg, [run.n], r, 3)
        parts.append(_run(M, [G], ns, c, per_particle=True))
    ev = torch.cat([o.events_pp for o in parts])
    X = torch.cat([o.X_pp for o in parts])
    assert torch.equal(ev, full.events_pp) and torch.equal(X, full.X_pp)
    for k in ("T", "q", "q_bin"):
        tot = sum(getattr(o, k) for o in parts)
        ref = getattr(full, k)
        assert torch.allclose(tot, ref, rtol=1e-12, atol=1e-12 * ref.abs().max().item()), k
    pooled = shard.combine_stats([o.stats[0].cpu().numpy() for o in parts])
    st = full.stats[0].cpu().numpy()
    assert pooled[L.STAT_N] == run.n and pooled[L.STAT_EVENTS] == st[L.STAT_EVENTS]
    assert pooled[L.STAT_KAPPA] == pytest.approx(st[L.STAT_KAPPA], rel=1e-12)
    assert pooled[L.STAT_KAPPA_SE] == pytest.approx(st[L.STAT_KAPPA_SE], rel=1e-9)
    with pytest.raises(L.MCBTEError):
        _run(M, [G], [10], replace(cfg, pid_begin=[run.n - 5], n_total=[run.n]))


def _exact_outputs(o):
    return [o.events_pp.cpu().numpy(), o.X_pp.cpu().numpy().view(np.int64), o.q_bin.cpu().numpy()]


def test_tail_draws_change_no_result():
    """The run's tail (warps with few particles left draw the next events of
    all of them at once) traces with the draws the inline path computes, so
    per-particle event counts, X_p and the fixed-point tallies are bit for bit
    those of runs without it, for every threshold and launch shape; with the
    two-phonon clock and internal walls (sub-block 256 draws) as well."""
    wl = W.film_batch_c4(scale=0.01)
    M = api.Material(wl.material)
    Gs = [api.Geometry(g) for g in wl.geometries]
    base = None
    for tail in (-1, 0, 3, 16, 32):
        for threads, refill in ((256, 1), (1024, 4)):
            cfg = api.SteadyConfig(seed=41, precision=L.FP32_TRACE, tally_axis=1, per_bin=True, n_scat_max=10,
                                   max_events=10 ** 8, threads_per_block=threads, refill_threshold=refill,
                                   tail_lanes=tail)
            o = _run(M, Gs, wl.n_per_geom, cfg, per_particle=True)
            assert np.all(o.stats[:, L.STAT_STATUS].cpu().numpy() == 0)
            cur = _exact_outputs(o)
            if base is None:
                base = cur
                continue
            for a, b in zip(cur, base):
                assert np.array_equal(a, b), (tail, threads)
    m = W.bvk_holland()
    m = replace(m, tau_imp=1.0 / (2e-44 * m.omega ** 4))
    M2, G2 = api.Material(m), api.Geometry(W.nanomesh())
    outs = []
    for tail in (-1, 8):
        cfg = api.SteadyConfig(seed=43, precision=L.FP32_TRACE, tally_axis=1, per_bin=True, n_scat_max=10,
                               max_events=10 ** 8, threads_per_block=512, tail_lanes=tail)
        outs.append(_exact_outputs(_run(M2, [G2], [200_000], cfg, per_particle=True)))
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def test_tail_draws_change_no_gradient():
    """The gradient's replay pass with the measure-valued d/dp_pore (its
    reservoir words come from the tail's draws too) gives the same gradient
    with and without the tail draws."""
    wl = W.pore_film_c5(n=300_000)
    M, G = api.Material(wl.material), api.Geometry(wl.geometries[0])
    res = []
    for tail in (-1, 0):
        cfg = api.SteadyConfig(seed=44, precision=L.FP32_TRACE, tally_axis=1, per_bin=True, n_scat_max=10,
                               max_events=10 ** 8, threads_per_block=768, refill_threshold=4, tail_lanes=tail)
        fwd, go = api.grad(M, G, wl.run.n, cfg)
        torch.cuda.synchronize()
        assert fwd.stats[0, L.STAT_STATUS].item() == 0
        res.append((fwd.q_bin.cpu().numpy(), go.dkappa_dlogtau.cpu().numpy(), go.dkappa_dp.cpu().numpy()))
    (q0, d0, p0), (q1, d1, p1) = res
    assert np.array_equal(q0, q1)
    # the resampling and specularity sums are FP64 atomics (order-dependent rounding)
    np.testing.assert_allclose(d1, d0, rtol=1e-12, atol=1e-12 * np.abs(d0).max())
    np.testing.assert_allclose(p1, p0, rtol=1e-9)


def test_graph_batch_replays_and_matches_direct_run():
    wl = W.film_batch_c4(n_films=8)
    mat, run = wl.material, wl.run
    M = api.Material(mat)
    Gs = [api.Geometry(g) for g in wl.geometries]
    ns = [3000, 100, 4500, 1, 800, 2500, 60, 1200]
    cfg = api.SteadyConfig(seed=77, precision=L.FP32_TRACE, tally_axis=1, per_bin=True, n_scat_max=10,
                           max_events=5_000_000)
    gb = batch.GraphBatch(M, Gs, ns, cfg, tune=False)
    a = gb.replay(seed=123)
    torch.cuda.synchronize()
    sa = a.stats.clone(); qa = a.q_bin.clone()
    gb.replay(seed=124)
    torch.cuda.synchronize()
    sb = gb.out.stats.clone()
    gb.replay(seed=123)
    torch.cuda.synchronize()
    assert torch.equal(gb.out.q_bin, qa)
    assert torch.allclose(gb.out.stats, sa, rtol=1e-12, atol=0)
    assert not torch.equal(sb[:, L.STAT_SUMX], sa[:, L.STAT_SUMX])
    direct = _run(M, Gs, ns, api.SteadyConfig(seed=123, precision=L.FP32_TRACE, tally_axis=1, per_bin=True,
                                              n_scat_max=10, max_events=5_000_000))
    assert torch.equal(direct.q_bin, qa)
    assert torch.allclose(direct.stats, sa, rtol=1e-12, atol=0)
    assert (sa[:, L.STAT_N].cpu().numpy() == np.array(ns)).all()


def test_graph_batch_with_detector_regions_matches_direct_run():
    """Detector regions reach the device as launch parameters, so a captured
    graph holds their bytes: replays (after the host list is gone) give the
    direct run's detector tallies bit for bit."""
    wl = W.si_slab_c2(n=50_000)
    mat, geo, run = wl.material, wl.geometries[0], wl.run
    M, G = api.Material(mat), api.Geometry(geo)
    Lb = geo.L
    regions = [((0.1 * Lb[0], 0.7 * Lb[0], 0.0, Lb[1], 0.25 * Lb[2], 0.75 * Lb[2]), (2, 2, 4)),
               ((0.0, Lb[0], 0.0, Lb[1], 0.0, Lb[2]), (1, 1, 8))]
    cfg = api.SteadyConfig(seed=5, precision=L.FP32_TRACE, tally_axis=2, per_bin=True, regions=regions)
    gb = batch.GraphBatch(M, [G], [run.n], cfg, tune=False)
    gb.replay(seed=777)
    gb.replay(seed=777)
    torch.cuda.synchronize()
    det_g, qb_g = gb.out.det.clone(), gb.out.q_bin.clone()
    d = _run(M, [G], [run.n], replace(cfg, seed=777))
    assert torch.equal(d.det, det_g) and torch.equal(d.q_bin, qb_g)
    assert torch.count_nonzero(det_g) > 0


def test_autotune_returns_a_valid_shape_with_the_same_physics():
    wl = W.si_slab_c2(n=200_000)
    mat, geo, run = wl.material, wl.geometries[0], wl.run
    M, G = api.Material(mat), api.Geometry(geo)
    cfg = api.SteadyConfig(seed=run.seed, precision=L.FP32_TRACE, n_cells=run.n_cells, tally_axis=2, per_bin=True)
    autotune.clear_cache()
    tuned = autotune.tune(M, [G], [run.n], cfg)
    assert tuned.threads_per_block in (256, 512, 768, 1024) and tuned.tail_lanes in (-1, 0)
    a = _run(M, [G], [run.n], cfg)
    b = _run(M, [G], [run.n], tuned)
    assert torch.equal(a.T, b.T) and torch.equal(a.q_bin, b.q_bin)
    assert autotune.tune(M, [G], [run.n], cfg) == tuned       # cached
    # the cache key holds what picks the kernel and its load: another
    # geometry, the two-phonon clock or the axis-only cell tallies are new keys
    key = autotune._key(M, [G], [run.n], cfg)
    geo2 = W.si_slab_c2(n=10).geometries[0]
    geo2.L = (2e-6, 2e-6, 1e-6)
    assert autotune._key(M, [api.Geometry(geo2)], [run.n], cfg) != key
    M2 = api.Material(replace(mat, tau_imp=1.0 / (2e-44 * mat.omega ** 4)))
    assert autotune._key(M2, [G], [run.n], cfg) != key
    assert autotune._key(M, [G], [run.n], replace(cfg, cell_flux_axis=True)) != key
    assert autotune._key(M, [G], [run.n], replace(cfg, nscat_curve=True)) != key
    # a tail threshold the caller set is kept
    assert autotune.tune(M, [G], [run.n], replace(cfg, tail_lanes=4)).tail_lanes == 4


def test_films_batched_kappa_vs_fuchs_sondheimer():
    wl = W.film_batch_c4(scale=0.05)
    mat, run = wl.material, wl.run
    tb = oracle.tables(mat)
    M = api.Material(mat)
    Gs = [api.Geometry(g) for g in wl.geometries]
    cfg = api.SteadyConfig(seed=1004, precision=L.FP32_TRACE, tally_axis=1, per_bin=True, n_scat_max=10,
                           max_events=200_000_000, time_budget_s=300)
    o = _run(M, Gs, wl.n_per_geom, cfg)
    st = o.stats.cpu().numpy()
    z = []
    for f, g in enumerate(wl.geometries):
        fs = cf.fuchs_sondheimer(tb["C"], mat.v, mat.tau, g.L[2])
        z.append((st[f, L.STAT_KAPPA] - fs) / st[f, L.STAT_KAPPA_SE])
    z = np.array(z)
    assert st[:, L.STAT_TRUNCATED].sum() == 0
    assert np.max(np.abs(z)) < 4.5, z
    assert np.mean(z ** 2) < 2.0, np.mean(z ** 2)


def test_autograd_backward_equals_library_gradient():
    mat = W.bvk_holland(n_per_branch=8)
    geo = W.pore_lattice(100e-9, 0.25, 200e-9, p_pore=0.3)
    cfg = api.SteadyConfig(seed=5, precision=L.FP32_TRACE, tally_axis=1, per_bin=False, n_scat_max=6,
                           max_events=5_000_000)
    s = torch.zeros(mat.n_bins, dtype=torch.float64, requires_grad=True)
    p = torch.tensor(0.3, dtype=torch.float64, requires_grad=True)
    k = autograd.kappa(s, p, mat, geo, 100_000, cfg)
    k.backward()
    _, go = api.grad(api.Material(mat), api.Geometry(geo), 100_000, cfg)
    torch.cuda.synchronize()
    assert torch.allclose(s.grad, go.dkappa_dlogtau.cpu(), rtol=1e-12, atol=0)
    assert p.grad.item() == pytest.approx(go.dkappa_dp[0].item(), rel=1e-12)


def _kappa_pp(mat, geo, cfg, n):
    o = _run(api.Material(mat), [api.Geometry(geo)], [n], cfg, per_particle=True)
    st = o.stats[0].cpu().numpy()
    X = o.X_pp.cpu().numpy()
    return st[L.STAT_KAPPA], st[L.STAT_KAPPA] / X.sum() * X


def test_autograd_gradient_matches_crn_central_differences():
    mat = W.bvk_holland(n_per_branch=8)
    geo = W.pore_lattice(100e-9, 0.25, 200e-9, p_pore=0.3)
    n = 1_000_000
    cfg = api.SteadyConfig(seed=11, precision=L.FP32_TRACE, tally_axis=1, n_scat_max=4, max_events=5_000_000)
    rng = np.random.default_rng(4)
    dirs = np.vstack([rng.choice([-1.0, 1.0], size=mat.n_bins), np.eye(mat.n_bins)[mat.n_bins - 3]])
    _, go = api.grad(api.Material(mat), api.Geometry(geo), n, cfg, dirs=dirs)
    torch.cuda.synchronize()
    lr = go.dkappa_dir[:2].cpu().numpy()
    h = 1e-2
    for k in range(2):
        kp, xp = _kappa_pp(mat.scaled_tau(h * dirs[k]), geo, cfg, n)
        km, xm = _kappa_pp(mat.scaled_tau(-h * dirs[k]), geo, cfg, n)
        fd = (kp - km) / (2 * h)
        fd_se = ((xp - xm) / (2 * h)).std(ddof=1) * math.sqrt(n)
        se = math.hypot(fd_se, lr[k, 1])
        assert abs(lr[k, 0] - fd) < 4 * se, (k, lr[k], fd, fd_se)
    # pore specularity
    gp = go.dkappa_dp.cpu().numpy()
    from dataclasses import replace
    kp, xp = _kappa_pp(mat, replace(geo, pore_p=0.3 + h), cfg, n)
    km, xm = _kappa_pp(mat, replace(geo, pore_p=0.3 - h), cfg, n)
    fd = (kp - km) / (2 * h)
    fd_se = ((xp - xm) / (2 * h)).std(ddof=1) * math.sqrt(n)
    assert abs(gp[0] - fd) < 4 * math.hypot(gp[1], fd_se), (gp, fd, fd_se)


def _timing_events(record=True):
    evs = tuple(torch.cuda.Event(enable_timing=True) for _ in range(2))
    if record:               # torch only reports elapsed time for events it recorded itself
        for e in evs:
            e.record()
        torch.cuda.synchronize()
    return evs


def _outer_ms(fn):
    a, b = _timing_events(record=False)
    a.record()
    fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b)


def test_trace_events_time_the_kernel_eagerly_and_in_graph_replays():
    wl = W.film_batch_c4(n_films=4)
    M = api.Material(wl.material)
    Gs = [api.Geometry(g) for g in wl.geometries]
    ns = [20_000] * len(Gs)
    evs = _timing_events()
    cfg = api.SteadyConfig(seed=5, precision=L.FP32_TRACE, tally_axis=1, per_bin=True, n_scat_max=10,
                           max_events=5_000_000, trace_events=evs)
    out = api.run_steady(M, Gs, ns, cfg)
    torch.cuda.synchronize()
    t_eager = evs[0].elapsed_time(evs[1])
    assert t_eager > 0.0
    assert (out.stats[:, L.STAT_N].cpu().numpy() == np.array(ns)).all()

    # events never recorded before the capture: the library must still get
    # real handles, and every replay must re-record the pair around the kernel
    gevs = _timing_events(record=False)
    gb = batch.GraphBatch(M, Gs, ns, replace_cfg(cfg, trace_events=gevs), tune=False)
    for seed in (11, 12):
        for e in gevs:
            e.record()
        step = _outer_ms(lambda: gb.replay(seed=seed))
        t = gevs[0].elapsed_time(gevs[1])
        assert 0.5 * step < t <= step, (t, step)

    wt = W.transient_box_c3(n=200_000)
    tevs = _timing_events()
    tr = wt.run
    tcfg = api.TransientConfig(seed=tr.seed, precision=L.FP32_TRACE, t_max=tr.t_max, t_meas=tr.t_meas,
                               grid=tr.grid, trace_events=tevs)
    api.run_transient(api.Material(wt.material), api.Geometry(wt.geometries[0]), tr.n, tcfg)
    torch.cuda.synchronize()
    assert tevs[0].elapsed_time(tevs[1]) > 0.0


def replace_cfg(cfg, **kw):
    from dataclasses import replace
    return replace(cfg, **kw)


def test_fp32_gradient_forward_equals_plain_run_and_is_reproducible():
    # the FP32 gradient's first pass is the plain forward run; the second
    # pass replays it, and its fixed-point gradient sums do not depend on
    # the order of the atomics
    wl = W.pore_film_c5(n=150_000, p_pore=0.4)
    mat, geo, run = wl.material, wl.geometries[0], wl.run
    M, G = api.Material(mat), api.Geometry(geo)
    cfg = api.SteadyConfig(seed=31, precision=L.FP32_TRACE, n_scat_max=run.n_scat_max, max_events=20_000_000,
                           tally_axis=run.tally_axis, per_bin=True, threads_per_block=512)
    f1, g1 = api.grad(M, G, run.n, cfg)
    plain = _run(M, [G], [run.n], cfg)
    f2, g2 = api.grad(M, G, run.n, replace_cfg(cfg, threads_per_block=1024, refill_threshold=8))
    torch.cuda.synchronize()
    assert f1.stats[0, L.STAT_STATUS].item() == 0 and f2.stats[0, L.STAT_STATUS].item() == 0
    assert torch.equal(f1.q_bin, plain.q_bin)
    assert f1.stats[0, L.STAT_EVENTS].item() == plain.stats[0, L.STAT_EVENTS].item()
    assert torch.equal(g1.dkappa_dlogtau, g2.dkappa_dlogtau)


@pytest.mark.parametrize("case", ["gauss_box", "walls", "two_phonon", "bin_average"])
def test_fp32_transient_time_windows_change_nothing(case):
    # windows hold whole flights and park particles at events, so any window
    # size reproduces the one-pass trajectories and integer tallies exactly
    if case == "bin_average":
        wl = W.transient_box_c3(n=300_000, grid=(16, 16, 8), n_times=23)
        wl.run.time_average = True
    elif case in ("gauss_box", "two_phonon"):
        wl = W.transient_box_c3(n=300_000, grid=(16, 16, 8), n_times=23)
        if case == "two_phonon":       # the parked state carries the two-phonon clock
            from dataclasses import replace
            wl.material = replace(wl.material, tau_imp=1.0 / (2e-44 * wl.material.omega ** 4))
    else:       # wall sources emit at t0 = R t_max; particles are absorbed mid-window
        wl = W.ballistic_transient_e1(n=300_000)
        wl.material.tau[:] = 20e-12
    r = wl.run
    M, G = api.Material(wl.material), api.Geometry(wl.geometries[0])
    nt = len(r.t_meas)
    outs = []
    for wt in (nt, 5, 1, 0):
        cfg = api.TransientConfig(seed=r.seed, t_max=r.t_max, t_meas=r.t_meas, grid=r.grid, precision=L.FP32_TRACE,
                                  window_times=wt, time_average=bool(getattr(r, "time_average", False)))
        o = api.run_transient(M, G, r.n, cfg, per_particle=True)
        torch.cuda.synchronize()
        assert o.stats[L.STAT_STATUS].item() == 0
        outs.append(o)
    base = outs[0]
    for o in outs[1:]:
        assert torch.equal(o.tally, base.tally)
        assert torch.equal(o.events_pp, base.events_pp)
        for k in (L.STAT_EVENTS, L.STAT_N, L.STAT_MAX_EVENTS, L.STAT_TRUNCATED):
            assert o.stats[k].item() == base.stats[k].item()
    assert base.stats[L.STAT_N].item() == r.n


def test_fp32_axis_only_cell_tallies_equal_the_full_ones():
    wl = W.si_slab_c2(n=200_000)
    mat, geo, run = wl.material, wl.geometries[0], wl.run
    M, G = api.Material(mat), api.Geometry(geo)
    cfg = api.SteadyConfig(seed=41, precision=L.FP32_TRACE, n_cells=run.n_cells, cell_axis=2, tally_axis=2,
                           per_bin=True)
    full = _run(M, [G], [run.n], cfg)
    axis = _run(M, [G], [run.n], replace_cfg(cfg, cell_flux_axis=True))
    assert torch.equal(axis.T, full.T)
    assert torch.equal(axis.q[..., 2], full.q[..., 2])
    assert torch.count_nonzero(axis.q[..., :2]) == 0
    assert torch.equal(axis.q_bin, full.q_bin)
    assert torch.equal(axis.stats[:, L.STAT_SUMX], full.stats[:, L.STAT_SUMX])


def test_l2_reduction_probe_adds_exactly():
    import bench
    slots = torch.zeros(4096, dtype=torch.int64, device="cuda")
    probe = bench.load_probe()
    s = torch.cuda.current_stream()
    assert probe.bench_l2_reduction_probe(slots.data_ptr(), 4096, 100_003, ctypes.c_void_p(s.cuda_stream)) == 0
    torch.cuda.synchronize()
    assert int(slots.sum().item()) == 4 * 100_003
    r = slots.view(-1, 4)
    assert torch.equal(r[:, 0], r[:, 3])          # the four words of a record move together
    assert int((r[:, 0] > 0).sum().item()) > 900   # the groups spread over the records


def test_fused_gradient_pass_equals_the_two_pass_replay():
    """With N_scat_max <= 16 and no cell tallies the FP32 gradient is one pass
    (each particle lists its periods' score sums until its final tally is
    known); asking for cell tallies makes it a forward pass plus a replay.
    Same particles, same trajectories: the forward tallies agree bit for bit,
    the gradient to the rounding of its split fixed-point terms, and the
    measure-valued d/dp (the same phantom tallies) to the order of its sums."""
    wl = W.pore_film_c5(n=200_000)
    mat, geo, run = wl.material, wl.geometries[0], wl.run
    M, G = api.Material(mat), api.Geometry(geo)
    base = api.SteadyConfig(seed=47, precision=L.FP32_TRACE, tally_axis=1, per_bin=True, n_scat_max=10,
                            max_events=10 ** 8, threads_per_block=512, refill_threshold=4)
    ones = np.ones((1, mat.n_bins))
    res = []
    for n_cells in (0, 4):
        fwd, go = api.grad(M, G, run.n, replace(base, n_cells=n_cells, cell_axis=2), dirs=ones)
        torch.cuda.synchronize()
        assert fwd.stats[0, L.STAT_STATUS].item() == 0
        res.append((fwd.q_bin.cpu().numpy(), fwd.stats[0].cpu().numpy(), go.dkappa_dlogtau.cpu().numpy(),
                    go.dkappa_dp.cpu().numpy(), go.dkappa_dir.cpu().numpy()))
    (q0, s0, d0, p0, r0), (q1, s1, d1, p1, r1) = res
    assert np.array_equal(q0, q1)
    assert s0[L.STAT_EVENTS] == s1[L.STAT_EVENTS]
    assert s0[L.STAT_KAPPA] == pytest.approx(s1[L.STAT_KAPPA], rel=1e-12)
    np.testing.assert_allclose(d0, d1, rtol=0, atol=1e-6 * np.abs(d1).max())
    assert d0.sum() == pytest.approx(d1.sum(), rel=1e-6)
    assert r0[0, 0] == pytest.approx(r1[0, 0], rel=1e-6)
    assert p0[0] == pytest.approx(p1[0], rel=1e-12) and p0[1] == pytest.approx(p1[1], rel=1e-9)


def test_unfolded_periodic_flights_keep_event_counts():
    """A forward flight without cell tallies runs through periodic faces and
    counts the crossings; with a cell tally the kernel stops at every face.
    The event counts agree particle by particle (a rare position that rounds
    onto a face may move one crossing), the tallies to rounding, kappa well
    within its standard error."""
    wl = W.film_batch_c4(n_films=8, scale=0.02)
    M = api.Material(wl.material)
    Gs = [api.Geometry(g) for g in wl.geometries]
    base = api.SteadyConfig(seed=53, precision=L.FP32_TRACE, tally_axis=1, per_bin=True, n_scat_max=10,
                            max_events=10 ** 8, threads_per_block=512, refill_threshold=4)
    unf = _run(M, Gs, wl.n_per_geom, base, per_particle=True)
    stp = _run(M, Gs, wl.n_per_geom, replace(base, n_cells=1, cell_axis=2), per_particle=True)
    e_u, e_s = unf.events_pp.cpu().numpy(), stp.events_pp.cpu().numpy()
    assert e_u.size == sum(wl.n_per_geom) and np.mean(e_u != e_s) < 1e-3
    same = e_u == e_s
    x_u, x_s = unf.X_pp.cpu().numpy(), stp.X_pp.cpu().numpy()
    assert np.max(np.abs(x_u[same] - x_s[same])) < 1e-3 * max(1.0, np.abs(x_s).max())
    su, ss = unf.stats.cpu().numpy(), stp.stats.cpu().numpy()
    assert np.all(su[:, L.STAT_STATUS] == 0) and np.all(ss[:, L.STAT_STATUS] == 0)
    z = (su[:, L.STAT_KAPPA] - ss[:, L.STAT_KAPPA]) / ss[:, L.STAT_KAPPA_SE]
    assert np.all(np.abs(z) < 0.5), z
