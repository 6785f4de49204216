"""Parity at the full workload sizes the bench times, in the launch
configurations it uses: the CPU reference traces the whole 1e7-particle slab
(16 host cores, a few seconds) or samples of particles one by one, and
properties that hold at any size (exact count conservation, invariance of
the integer tallies under time windows, the gradient against common-random-
number central differences) cover the rest."""
from dataclasses import replace

import numpy as np
import pytest

import oracle
from inputs import workloads as W
from gpu_helpers import rel_close

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2104_03573_gb300 import _lib as L  # noqa: E402
from paper_2104_03573_gb300 import api, batch  # noqa: E402

RTOL = 1e-9


def _ranges(n, k, width, seed):
    """k runs of `width` consecutive particle ids spread over [0, n), plus both ends."""
    rng = np.random.default_rng(seed)
    starts = np.unique(np.concatenate([[0, n - width], rng.integers(0, n - width, size=k)]))
    return [(int(s), int(s) + width) for s in starts]


def _oracle_sample(mat, geom, run, n_total, ranges, batch_index=0):
    ev, X = [], []
    for a, b in ranges:
        r = oracle.run_steady(mat, geom, run, pid_begin=a, pid_end=b, n_total=n_total, batch_index=batch_index,
                              per_particle=True, n_threads=1)
        ev.append(r["events_pp"])
        X.append(r["X_pp"])
    return np.concatenate(ev), np.concatenate(X)


def _take(arr, ranges):
    return np.concatenate([arr[a:b] for a, b in ranges])


def test_si_slab_full_size_fp64_tallies_and_fp32_kappa():
    wl = W.si_slab_c2()                                   # 1e7 particles, 50 cells + per-bin flux
    mat, geo, run = wl.material, wl.geometries[0], wl.run
    ref = oracle.run_steady(mat, geo, run)                # all particles, all host cores
    M, G = api.Material(mat), api.Geometry(geo)
    base = dict(seed=run.seed, n_cells=run.n_cells, cell_axis=run.cell_axis, tally_axis=run.tally_axis,
                per_bin=True, max_events=run.max_events)
    f64 = api.run_steady(M, [G], [run.n], api.SteadyConfig(precision=L.FP64_PLAIN, **base))
    torch.cuda.synchronize()
    for k, ours in (("T", f64.T[0]), ("q", f64.q[0]), ("q_bin", f64.q_bin[0])):
        ok, err = rel_close(ours.cpu().numpy(), ref[k], RTOL)
        assert ok, (k, err)
    st = f64.stats[0].cpu().numpy()
    assert st[L.STAT_EVENTS] == ref["events"]
    assert st[L.STAT_KAPPA] == pytest.approx(ref["kappa"], rel=RTOL)
    # FP32 tracer in the bench's launch shapes, same random words
    for threads, refill in ((1024, 4), (768, 4)):
        o = api.run_steady(M, [G], [run.n], api.SteadyConfig(precision=L.FP32_TRACE, threads_per_block=threads,
                                                             refill_threshold=refill, **base))
        torch.cuda.synchronize()
        s32 = o.stats[0].cpu().numpy()
        assert s32[L.STAT_STATUS] == 0 and s32[L.STAT_N] == run.n
        se = np.hypot(s32[L.STAT_KAPPA_SE], ref["kappa_se"])
        assert abs(s32[L.STAT_KAPPA] - ref["kappa"]) < min(3 * se, 0.005 * ref["kappa"])


def test_si_slab_full_size_sampled_particles():
    wl = W.si_slab_c2()
    mat, geo, run = wl.material, wl.geometries[0], wl.run
    M, G = api.Material(mat), api.Geometry(geo)
    o = api.run_steady(M, [G], [run.n], api.SteadyConfig(seed=run.seed, precision=L.FP64_PLAIN, n_cells=run.n_cells,
                                                         tally_axis=run.tally_axis, per_bin=True,
                                                         max_events=run.max_events), per_particle=True)
    torch.cuda.synchronize()
    ranges = _ranges(run.n, 24, 16, 11)
    ev, X = _oracle_sample(mat, geo, run, run.n, ranges)
    assert np.array_equal(_take(o.events_pp.cpu().numpy().astype(np.uint32), ranges), ev)
    # X_p bit for bit: one thread's sum of the same IEEE operations on both sides
    assert np.array_equal(_take(o.X_pp.cpu().numpy(), ranges).view(np.int64), X.view(np.int64))


def test_transient_box_full_size_counts_and_windows():
    wl = W.transient_box_c3()                             # 1e8 particles, 64x64x32 cells x 200 times
    mat, geo, run = wl.material, wl.geometries[0], wl.run
    M, G = api.Material(mat), api.Geometry(geo)
    out = api.TransientOutputs(len(run.t_meas), run.grid, run.n)
    outs = []
    for wt in (0, len(run.t_meas)):                       # the bench's windows, then one pass
        cfg = api.TransientConfig(seed=run.seed, t_max=run.t_max, t_meas=run.t_meas, grid=run.grid,
                                  precision=L.FP32_TRACE, window_times=wt)
        api.run_transient(M, G, run.n, cfg, out=out)
        torch.cuda.synchronize()
        st = out.stats.cpu().numpy()
        assert st[L.STAT_STATUS] == 0 and st[L.STAT_N] == run.n
        outs.append((out.tally.clone(), st))
    assert torch.equal(outs[0][0], outs[1][0])
    assert outs[0][1][L.STAT_EVENTS] == outs[1][1][L.STAT_EVENTS]
    # every particle is inside the adiabatic box at every measurement time and
    # every sign is +: each snapshot's temperature field sums to N quanta of
    # E_eff / (C_tot V_cell) (Eq. sampling)
    ncell = run.grid[0] * run.grid[1] * run.grid[2]
    v_cell = float(np.prod(geo.L)) / ncell
    quantum = (outs[0][1][L.STAT_E_TOT] / run.n) / (M.tables()["C_tot"] * v_cell)
    per_time = (outs[0][0][..., 0].sum(dim=(1, 2, 3)) / quantum).cpu().numpy()
    np.testing.assert_allclose(per_time, run.n, rtol=1e-9)


def test_film_batch_full_size_sampled_particles_and_fp32_batch():
    wl = W.film_batch_c4()                                # 64 films, ~1.4e8 particles
    mat, run = wl.material, wl.run
    ns = list(wl.n_per_geom)
    M = api.Material(mat)
    Gs = [api.Geometry(g) for g in wl.geometries]
    base = dict(tally_axis=run.tally_axis, per_bin=True, n_scat_max=run.n_scat_max, max_events=10 ** 9,
                time_budget_s=300)
    f64 = api.run_steady(M, Gs, ns, api.SteadyConfig(seed=run.seed, precision=L.FP64_PLAIN, **base),
                         per_particle=True)
    torch.cuda.synchronize()
    st64 = f64.stats.cpu().numpy()
    assert np.all(st64[:, L.STAT_STATUS] == 0)
    ev_all = f64.events_pp.cpu().numpy().astype(np.uint32)
    X_all = f64.X_pp.cpu().numpy()
    off = np.concatenate([[0], np.cumsum(ns)])
    for f in (0, 1, 9, 21, 40, 63):
        rr = _ranges(ns[f], 3, 8, 100 + f)
        ev, X = _oracle_sample(mat, wl.geometries[f], run, ns[f], rr, batch_index=f)
        glob = [(a + off[f], b + off[f]) for a, b in rr]
        assert np.array_equal(_take(ev_all, glob), ev), f
        assert np.array_equal(_take(X_all, glob).view(np.int64), X.view(np.int64)), f
    # FP32: the bench's batched launch (CUDA graph, device-resident key)
    gb = batch.GraphBatch(M, Gs, ns, api.SteadyConfig(seed=run.seed, precision=L.FP32_TRACE, **base), tune=True)
    o = gb.replay(seed=run.seed)
    torch.cuda.synchronize()
    st = o.stats.cpu().numpy()
    assert np.all(st[:, L.STAT_STATUS] == 0)
    assert np.array_equal(st[:, L.STAT_N], np.array(ns, dtype=np.float64))
    z = (st[:, L.STAT_KAPPA] - st64[:, L.STAT_KAPPA]) / np.hypot(st[:, L.STAT_KAPPA_SE], st64[:, L.STAT_KAPPA_SE])
    assert np.all(np.abs(z) < 3.0), z


def test_pore_grad_full_size_replay_and_crn_differences():
    wl = W.pore_film_c5()                                 # 5e7 particles
    mat, geo, run = wl.material, wl.geometries[0], wl.run
    M, G = api.Material(mat), api.Geometry(geo)
    cfg = api.SteadyConfig(seed=run.seed, precision=L.FP32_TRACE, tally_axis=run.tally_axis, per_bin=True,
                           n_scat_max=run.n_scat_max, max_events=10 ** 9, threads_per_block=768,
                           refill_threshold=4, time_budget_s=300)
    ones = np.ones((1, mat.n_bins))
    fwd, go = api.grad(M, G, run.n, cfg, dirs=ones)
    torch.cuda.synchronize()
    assert fwd.stats[0, L.STAT_STATUS].item() == 0       # no truncation, no time-out (one fused pass)
    d, d_se = go.dkappa_dir[0].cpu().numpy()
    # common random numbers: kappa(tau e^{+h}) - kappa(tau e^{-h}) over 2h,
    # with its own standard error from the per-particle differences (the two
    # runs share their random words but not every trajectory)
    h = 0.05
    ks, xs = [], []
    for sgn in (1.0, -1.0):
        m2 = replace(mat, tau=mat.tau * np.exp(sgn * h))
        o = api.run_steady(api.Material(m2), [G], [run.n], cfg, per_particle=True)
        torch.cuda.synchronize()
        ks.append(o.stats[0, L.STAT_KAPPA].item())
        xs.append(o.X_pp)
    fd = (ks[0] - ks[1]) / (2 * h)
    dpp = (xs[0] - xs[1]) / (2 * h)
    fd_se = abs(ks[0] / xs[0].sum().item()) * dpp.std().item() * np.sqrt(run.n)
    assert abs(d - fd) < 4 * np.hypot(d_se, fd_se) + 0.002 * abs(fd), (d, d_se, fd, fd_se)


def test_pore_grad_full_size_lr_against_crn_differences():
    """The likelihood-ratio gradient of the pore film at its configured size
    (3000 log-tau scales, 5e7 particles, diffuse pores) against central
    differences with common random numbers at h = 1e-3 and 2e-3 (the step
    halved and doubled shows the bias of non-smooth event switches), along 8
    random +-1 directions and 16 single bins (those with the largest gradient
    on an independent run), and the measure-valued d kappa / d p_pore at
    p = 0 against the one-sided second-order CRN quotient (p = 0, 1e-3,
    2e-3).  Every comparison is a z-test with both standard errors (the
    difference quotient's from its per-particle differences); 49 comparisons,
    so |z| < 4.5 bounds the family-wise false alarms near 3e-4.  At this size
    the difference quotients carry standard errors 30-100 times the
    likelihood ratio's (trajectory switches make their variance grow as 1/h),
    so they bound the gradient rather than resolve it."""
    wl = W.pore_film_c5()
    mat, geo, run = wl.material, wl.geometries[0], wl.run
    N = run.n
    G = api.Geometry(geo)
    cfg = api.SteadyConfig(seed=run.seed, precision=L.FP32_TRACE, tally_axis=1, per_bin=True, n_scat_max=10,
                           max_events=10 ** 9, threads_per_block=768, refill_threshold=4, time_budget_s=300)
    nb = mat.n_bins
    rand = np.random.default_rng(2104).choice([-1.0, 1.0], size=(8, nb))
    _, g0 = api.grad(api.Material(mat), G, N, replace(cfg, seed=run.seed + 100))
    bins = np.argsort(-np.abs(g0.dkappa_dlogtau.cpu().numpy()))[:16]
    dirs = np.concatenate([rand, np.eye(nb)[bins]])
    M = api.Material(mat)
    lr = []
    for k in range(0, 24, 12):
        _, go = api.grad(M, G, N, cfg, dirs=dirs[k:k + 12])
        lr.append(go.dkappa_dir.cpu().numpy())
    lr = np.concatenate(lr)

    def kappa_and_x(m, g=G):
        o = api.run_steady(api.Material(m) if m is not None else M, [g], [N], cfg, per_particle=True)
        torch.cuda.synchronize()
        return o.stats[0, L.STAT_KAPPA].item(), o.stats[0, L.STAT_SUMX].item(), o.X_pp.clone()

    z = []
    for k in range(24):
        for h in (1e-3, 2e-3):
            kp, sxp, xp = kappa_and_x(replace(mat, tau=mat.tau * np.exp(h * dirs[k])))
            km, _, xm = kappa_and_x(replace(mat, tau=mat.tau * np.exp(-h * dirs[k])))
            fd = (kp - km) / (2 * h)
            fd_se = abs(kp / sxp) * ((xp - xm) / (2 * h)).std().item() * np.sqrt(N)
            z.append((lr[k, 0] - fd) / np.hypot(lr[k, 1], fd_se))
    _, go = api.grad(M, G, N, cfg)
    mvd, mvd_se = go.dkappa_dp.cpu().numpy()
    ks, xs = [], []
    for p in (0.0, 1e-3, 2e-3):
        k_, sx_, x_ = kappa_and_x(None, api.Geometry(replace(geo, pore_p=p)))
        ks.append(k_)
        xs.append(x_)
    fd = (-3 * ks[0] + 4 * ks[1] - ks[2]) / 2e-3
    fd_se = abs(ks[2] / sx_) * ((-3 * xs[0] + 4 * xs[1] - xs[2]) / 2e-3).std().item() * np.sqrt(N)
    z.append((mvd - fd) / np.hypot(mvd_se, fd_se))
    z = np.array(z)
    assert np.all(np.isfinite(z)) and np.max(np.abs(z)) < 4.5, z
    assert np.mean(z ** 2) < 2.0, z
