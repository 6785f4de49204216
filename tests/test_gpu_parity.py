"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

FP64 plain mode: per-particle event counts identical; per-particle X_p bit
for bit (each is one thread's sum of the same IEEE operations in the same
order on both sides); every tally within 1e-9 of the oracle relative to the
tally's largest magnitude (tallies are sums of atomics whose order differs
run to run, and a signed sum can cancel below its terms).  FP32 mode: every
compared tally within 3 combined standard errors of the oracle on
independent seeds, kappa within 0.5 %.
"""
from dataclasses import replace

import numpy as np
import pytest

import oracle
from oracle import closed_forms as cf
from inputs import workloads as W
from gpu_helpers import batch_stats, gpu_steady, gpu_transient, rel_close, z_scores

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2104_03573_gb300 import _lib as L  # noqa: E402
from paper_2104_03573_gb300 import api  # noqa: E402

RTOL = 1e-9


def _check_fp64(g, ref, mask_events=True, tallies=("T", "q")):
    ev_ok = np.array_equal(g["events_pp"], ref["events_pp"])
    n_bad = int(np.sum(g["events_pp"] != ref["events_pp"]))
    assert ev_ok, f"{n_bad} particles with different event counts"
    a = np.ascontiguousarray(g["X_pp"], dtype=np.float64)
    b = np.ascontiguousarray(ref["X_pp"], dtype=np.float64)
    n_diff = int(np.sum(a.view(np.int64) != b.view(np.int64)))
    assert n_diff == 0, f"{n_diff} particles whose X_p differs from the oracle's in some bit"
    for k in tallies:
        if k in ref and k in g:
            ok, err = rel_close(g[k].reshape(ref[k].shape), ref[k], RTOL)
            assert ok, f"{k} rel err {err}"


# ------------------------------------------------------------------ tables (a1)
def test_tables_match_oracle_format2():
    m = W.gray(6000.0, 100e-9)
    rng = np.random.default_rng(0)
    n = 1000
    m = W.Material(omega=np.linspace(1e12, 7e13, n), v=rng.uniform(1e3, 9e3, n), tau=10 ** rng.uniform(-12, -9, n),
                   C=rng.exponential(size=n) * 1e3, T_lin=300.0)
    t_g = api.Material(m).tables()
    t_o = oracle.tables(m)
    assert np.array_equal(t_g["C"], t_o["C"])
    assert np.array_equal(t_g["alias"], t_o["alias"])
    assert np.array_equal(t_g["thr"], t_o["thr"])
    assert np.array_equal(t_g["prob"], t_o["prob"])
    assert t_g["sum_Cv"] == t_o["sum_Cv"] and t_g["C_tot"] == t_o["C_tot"]


def test_tables_match_oracle_bvk_format1():
    m = W.bvk_holland()
    t_g = api.Material(m).tables()
    t_o = oracle.tables(m)
    ok, err = rel_close(t_g["C"], t_o["C"], 1e-14)
    assert ok, err
    assert np.array_equal(t_g["alias"], t_o["alias"])
    d = np.abs(t_g["thr"].astype(np.float64) - t_o["thr"].astype(np.float64)) / 2.0 ** 64
    assert d.max() < 1e-12


# ------------------------------------------------------------------ FP64 parity
def test_fp64_gray_slab_full_size():
    wl = W.gray_slab_c1()                           # full size: 1e5 particles, 50 cells
    mat, g, run = wl.material, wl.geometries[0], wl.run
    gg = gpu_steady(mat, [g], [run.n], run, L.FP64_PLAIN, per_particle=True)
    ref = oracle.run_steady(mat, g, run, per_particle=True)
    _check_fp64({"events_pp": gg["events_pp"], "X_pp": gg["X_pp"], "T": gg["T"][0], "q": gg["q"][0]}, ref)
    st = gg["stats"][0]
    assert st[L.STAT_KAPPA] == pytest.approx(ref["kappa"], rel=RTOL)
    assert st[L.STAT_EVENTS] == ref["events"]
    assert st[L.STAT_SIGNED_ABSORBED] == st[L.STAT_SIGNED_EMITTED]


def test_fp64_against_an_oracle_with_library_transcendentals():
    """The FP64 path against the oracle evaluating ln, sin and cos with the C
    library (not the fixed series both sides share): slab particles keep
    their event counts (X_p to rounding); in the pore lattice a small fraction
    of trajectories part ways where diffuse pore reflections amplify last-bit
    differences, and the estimates agree within their standard errors."""
    wl = W.si_slab_c2(n=20_000)
    mat, g, run = wl.material, wl.geometries[0], wl.run
    gg = gpu_steady(mat, [g], [run.n], run, L.FP64_PLAIN, per_particle=True)
    with oracle.libm_mode():
        ref = oracle.run_steady(mat, g, run, per_particle=True)
    assert np.array_equal(gg["events_pp"], ref["events_pp"])
    assert np.max(np.abs(gg["X_pp"] - ref["X_pp"])) <= 1e-9 * 1000.0      # nm; the slab is 1 um
    wl = W.pore_film_c5(n=20_000)
    mat, g, run = wl.material, wl.geometries[0], wl.run
    run.max_events = 20_000_000
    gg = gpu_steady(mat, [g], [run.n], run, L.FP64_PLAIN, per_particle=True)
    with oracle.libm_mode():
        ref = oracle.run_steady(mat, g, run, per_particle=True)
    frac = np.mean(gg["events_pp"] != ref["events_pp"])
    assert frac < 0.02, frac
    st = gg["stats"][0]
    assert abs(st[L.STAT_KAPPA] - ref["kappa"]) < 3.0 * np.hypot(st[L.STAT_KAPPA_SE], ref["kappa_se"])


def test_fp64_bvk_slab_per_bin():
    wl = W.si_slab_c2(n=20_000)
    mat, g, run = wl.material, wl.geometries[0], wl.run
    gg = gpu_steady(mat, [g], [run.n], run, L.FP64_PLAIN, per_particle=True)
    ref = oracle.run_steady(mat, g, run, per_particle=True)
    _check_fp64({"events_pp": gg["events_pp"], "X_pp": gg["X_pp"], "T": gg["T"][0], "q": gg["q"][0],
                 "q_bin": gg["q_bin"][0]}, ref, tallies=("T", "q", "q_bin"))


def _with_imp(m, law=lambda w: 1.0 / (2e-44 * w ** 4)):
    return replace(m, tau_imp=np.asarray(law(np.asarray(m.omega, dtype=np.float64)), dtype=np.float64))


def test_fp64_two_phonon_clock_slab_per_particle():
    # separate two- and three-phonon clocks (Sec. 3.3) with the paper's
    # impurity law; a few bins without impurity scattering (+inf)
    wl = W.si_slab_c2(n=20_000)
    g, run = wl.geometries[0], wl.run
    mat = _with_imp(wl.material)
    mat.tau_imp[::97] = np.inf
    gg = gpu_steady(mat, [g], [run.n], run, L.FP64_PLAIN, per_particle=True)
    ref = oracle.run_steady(mat, g, run, per_particle=True)
    _check_fp64({"events_pp": gg["events_pp"], "X_pp": gg["X_pp"], "T": gg["T"][0], "q": gg["q"][0],
                 "q_bin": gg["q_bin"][0]}, ref, tallies=("T", "q", "q_bin"))
    plain = oracle.run_steady(wl.material, g, run, per_particle=True)
    assert ref["events"] > 1.05 * plain["events"]          # the clock adds events


def test_fp64_two_phonon_clock_transient_and_gradient():
    wl = W.transient_box_c3(n=3000, grid=(16, 16, 8), n_times=20)
    g, run = wl.geometries[0], wl.run
    mat = _with_imp(wl.material)
    gg = gpu_transient(mat, g, run, L.FP64_PLAIN, per_particle=True)
    ref = oracle.run_transient(mat, g, run, per_particle=True)
    assert np.array_equal(gg["events_pp"], ref["events_pp"])
    ok, err = rel_close(gg["tally"], ref["tally"], RTOL)
    assert ok, err
    # gradient: flights ended by the two-phonon clock are censored for tau
    wp = W.pore_film_c5(n=3000, p_pore=0.3)
    gp, rp = wp.geometries[0], wp.run
    rp.max_events = 2_000_000
    mp = _with_imp(wp.material)
    cfg = api.SteadyConfig(seed=rp.seed, precision=L.FP64_PLAIN, n_scat_max=rp.n_scat_max,
                           max_events=rp.max_events, tally_axis=rp.tally_axis, per_bin=True)
    fwd, go = api.grad(api.Material(mp), api.Geometry(gp), rp.n, cfg)
    torch.cuda.synchronize()
    rg = oracle.run_steady(mp, gp, rp, grad=True)
    ok, err = rel_close(go.dkappa_dlogtau.cpu().numpy(), rg["dkappa_dlogtau"], RTOL)
    assert ok, err
    assert fwd.stats[0, L.STAT_KAPPA].item() == pytest.approx(rg["kappa"], rel=RTOL)


def test_fp32_two_phonon_clock_kappa_vs_oracle():
    wl = W.pore_film_c5(n=300_000)
    g, run = wl.geometries[0], wl.run
    mat = _with_imp(wl.material)
    run.max_events = 10 ** 8
    gg = gpu_steady(mat, [g], [run.n], run, L.FP32_TRACE, seed=901)
    ref = oracle.run_steady(mat, g, run)
    k, se = gg["stats"][0][L.STAT_KAPPA], gg["stats"][0][L.STAT_KAPPA_SE]
    assert gg["stats"][0][L.STAT_STATUS] == 0
    assert abs(k - ref["kappa"]) < 3.5 * np.hypot(se, ref["kappa_se"])
    plain = oracle.run_steady(wl.material, g, run)
    assert ref["kappa"] < plain["kappa"] - 5 * np.hypot(ref["kappa_se"], plain["kappa_se"])


def _nanomesh_case(n, spec_low=False):
    # the paper's nanomesh (Sec. 5.5): 34 nm cell, 11 nm square pore through a
    # 22 nm film, diffuse walls, tau_imp^-1 = 2e-44 omega^4, N_scat^max = 10;
    # spec_low: modes up to 2 THz reflect specularly from every wall
    m = _with_imp(W.bvk_holland())
    g = W.nanomesh()
    if spec_low:
        m = replace(m, spec_bin=(m.omega / (2 * np.pi) <= 2e12).astype(np.float64))
        g.inner_p = [-1.0] * 4
        g.face_p = [(-1.0 if t == W.ADIABATIC else 0.0) for t in g.face_type]
    run = W.SteadyRun(n=n, seed=1006, tally_axis=1, per_bin=True, n_scat_max=10, max_events=10 ** 8)
    return m, g, run


@pytest.mark.parametrize("spec_low", [False, True])
def test_fp64_nanomesh_internal_walls_per_particle(spec_low):
    m, g, run = _nanomesh_case(3000, spec_low)
    gg = gpu_steady(m, [g], [run.n], run, L.FP64_PLAIN, per_particle=True)
    ref = oracle.run_steady(m, g, run, per_particle=True)
    _check_fp64({"events_pp": gg["events_pp"], "X_pp": gg["X_pp"], "q_bin": gg["q_bin"][0]}, ref,
                tallies=("q_bin",))
    assert gg["stats"][0][L.STAT_KAPPA] == pytest.approx(ref["kappa"], rel=RTOL)


def test_fp32_nanomesh_kappa_vs_oracle():
    m, g, run = _nanomesh_case(200_000)
    gg = gpu_steady(m, [g], [run.n], run, L.FP32_TRACE, seed=902)
    ref = oracle.run_steady(m, g, run)
    s = gg["stats"][0]
    assert s[L.STAT_STATUS] == 0
    assert abs(s[L.STAT_KAPPA] - ref["kappa"]) < 3.5 * np.hypot(s[L.STAT_KAPPA_SE], ref["kappa_se"])
    ms, gs, _ = _nanomesh_case(200_000, spec_low=True)
    gsp = gpu_steady(ms, [gs], [run.n], run, L.FP32_TRACE, seed=903)
    assert gsp["stats"][0][L.STAT_KAPPA] > s[L.STAT_KAPPA] + 4 * np.hypot(gsp["stats"][0][L.STAT_KAPPA_SE],
                                                                           s[L.STAT_KAPPA_SE])


def test_fp64_and_fp32_diagonal_control_gradient():
    # control gradient with several components (Lambertian frame about grad T)
    wl = W.pore_film_c5(n=4000)
    m, g, run = wl.material, wl.geometries[0], wl.run
    g.grad_T = (-0.6e6, -0.8e6, 0.0)
    run.max_events = 10 ** 8
    gg = gpu_steady(m, [g], [run.n], run, L.FP64_PLAIN, per_particle=True)
    ref = oracle.run_steady(m, g, run, per_particle=True)
    _check_fp64({"events_pp": gg["events_pp"], "X_pp": gg["X_pp"], "q_bin": gg["q_bin"][0]}, ref,
                tallies=("q_bin",))
    mg = W.gray(6000.0, 100e-9, C=1e6)
    gb = W.film(1e-6)
    gb.face_type = [W.PERIODIC] * 6
    gb.grad_T = (-1e6 / np.sqrt(2), -1e6 / np.sqrt(2), 0.0)
    rb = W.SteadyRun(n=1_000_000, seed=45, tally_axis=0, n_scat_max=3)
    g32 = gpu_steady(mg, [gb], [rb.n], rb, L.FP32_TRACE)
    k = cf.kinetic_kappa([1e6], [6000.0], [100e-9 / 6000.0])
    s32 = g32["stats"][0]
    assert abs(s32[L.STAT_KAPPA] - k) < 3.5 * s32[L.STAT_KAPPA_SE]


def test_detector_regions_fp64_parity_and_fp32_identities():
    # Sec. 4.5 regions: a coarse region, the same region split 4 x 4 x 4, and
    # two halves tiling the box
    box = (0.5e-6, 1.5e-6, 0.4e-6, 1.7e-6, 0.3e-6, 1.0e-6)
    halves = [((0.0, 1e-6, 0.0, 2e-6, 0.0, 1e-6), (2, 3, 2)), ((1e-6, 2e-6, 0.0, 2e-6, 0.0, 1e-6), (5, 1, 2))]
    wl = W.transient_box_c3(n=3000, grid=(8, 8, 4), n_times=12)
    m, g, run = wl.material, wl.geometries[0], wl.run
    run.regions = [(box, (1, 1, 1)), (box, (4, 4, 4))] + halves
    gg = gpu_transient(m, g, run, L.FP64_PLAIN, per_particle=True)
    ref = oracle.run_transient(m, g, run, per_particle=True)
    assert np.array_equal(gg["events_pp"], ref["events_pp"])
    ok, err = rel_close(gg["tally"], ref["tally"], RTOL)
    assert ok, err
    run.n = 400_000
    f32 = gpu_transient(m, g, run, L.FP32_TRACE)
    T = f32["tally"][..., 0]
    q = ref["V_cell"]                                 # per-detector volumes
    quanta = f32["stats"][L.STAT_E_TOT] / run.n / (oracle.tables(m)["C_tot"] * q)
    cnt = np.rint(T / quanta[None, :])
    assert np.array_equal(cnt[:, 0], cnt[:, 1:65].sum(axis=1))       # refined = coarse, exactly
    assert np.all(cnt[:, 65:].sum(axis=1) == run.n)                  # tiling halves count everyone


@pytest.mark.parametrize("with_regions", [False, True])
def test_time_bin_averages_fp64_parity_and_fp32_conservation(with_regions):
    wl = W.transient_box_c3(n=3000, grid=(8, 8, 4), n_times=12)
    m, g, run = wl.material, wl.geometries[0], wl.run
    run.time_average = True
    if with_regions:
        box = (0.5e-6, 1.5e-6, 0.4e-6, 1.7e-6, 0.3e-6, 1.0e-6)
        run.regions = [(box, (4, 4, 4)), ((0.0, 2e-6, 0.0, 2e-6, 0.0, 1e-6), (3, 5, 2))]
    gg = gpu_transient(m, g, run, L.FP64_PLAIN, per_particle=True)
    ref = oracle.run_transient(m, g, run, per_particle=True)
    assert np.array_equal(gg["events_pp"], ref["events_pp"])
    ok, err = rel_close(gg["tally"], ref["tally"], RTOL)
    assert ok, err
    run.n = 400_000
    f32 = gpu_transient(m, g, run, L.FP32_TRACE)
    assert f32["stats"][L.STAT_STATUS] == 0
    T = f32["tally"][..., 0].reshape(len(run.t_meas), -1)
    vd = np.broadcast_to(np.asarray(ref["V_cell"], dtype=np.float64), T.shape[1:])
    quanta = f32["stats"][L.STAT_E_TOT] / run.n / (oracle.tables(m)["C_tot"] * vd)
    cnt = T / quanta[None, :]
    whole = cnt if not with_regions else cnt[:, 64:]
    np.testing.assert_allclose(whole.sum(axis=1), run.n, rtol=1e-6)   # every particle, every whole bin


def test_steady_detector_regions_fp64_parity_and_fp32():
    wl = W.si_slab_c2(n=20_000)
    m, g, run = wl.material, wl.geometries[0], wl.run
    Lb = g.L
    sub = ((0.1 * Lb[0], 0.7 * Lb[0], 0.0, Lb[1], 0.25 * Lb[2], 0.75 * Lb[2]), (2, 2, 4))
    slabs = ((0.0, Lb[0], 0.0, Lb[1], 0.0, Lb[2]), (1, 1, run.n_cells))
    run.regions = [slabs, sub]
    M, G = api.Material(m), api.Geometry(g)
    base = dict(seed=run.seed, n_cells=run.n_cells, cell_axis=2, tally_axis=2, per_bin=True,
                max_events=run.max_events, regions=run.regions)
    o = api.run_steady(M, [G], [run.n], api.SteadyConfig(precision=L.FP64_PLAIN, **base))
    torch.cuda.synchronize()
    ref = oracle.run_steady(m, g, run)
    ok, err = rel_close(o.det[:, 0].cpu().numpy(), ref["det_T"], RTOL)
    assert ok, err
    ok, err = rel_close(o.det[:, 1:].cpu().numpy(), ref["det_q"], RTOL)
    assert ok, err
    # FP32: the slab slices of the region equal the 1-D cell tallies statistically
    o32 = api.run_steady(M, [G], [1_000_000], api.SteadyConfig(precision=L.FP32_TRACE, **base))
    torch.cuda.synchronize()
    d = o32.det.cpu().numpy()
    nc = run.n_cells
    T1 = o32.T[0].cpu().numpy()
    assert np.max(np.abs(d[:nc, 0] - T1)) < 1e-3 * np.max(np.abs(T1)) + 1e-6
    assert abs(d[nc:, 0].mean() - ref["det_T"][nc:].mean()) < 0.1 * np.abs(ref["det_T"]).max()


def test_fp64_film_batch_geometry_index_streams():
    wl = W.film_batch_c4(n_films=6)
    mat = wl.material
    run = wl.run
    run.max_events = 2_000_000
    ns = [700, 1, 333, 1000, 257, 64]                # ragged, includes a single particle
    geoms = wl.geometries
    gg = gpu_steady(mat, geoms, ns, run, L.FP64_PLAIN, per_particle=True)
    off = np.concatenate([[0], np.cumsum(ns)])
    for f in range(len(ns)):
        ref = oracle.run_steady(mat, geoms[f], run, n_total=ns[f], batch_index=f, per_particle=True)
        sl = slice(off[f], off[f + 1])
        _check_fp64({"events_pp": gg["events_pp"][sl], "X_pp": gg["X_pp"][sl], "q_bin": gg["q_bin"][f]}, ref,
                    tallies=("q_bin",))
        assert gg["stats"][f][L.STAT_KAPPA] == pytest.approx(ref["kappa"], rel=RTOL, abs=1e-12)


def test_fp64_pore_lattice():
    wl = W.pore_film_c5(n=5000)
    mat, g, run = wl.material, wl.geometries[0], wl.run
    run.max_events = 2_000_000
    gg = gpu_steady(mat, [g], [run.n], run, L.FP64_PLAIN, per_particle=True)
    ref = oracle.run_steady(mat, g, run, per_particle=True)
    _check_fp64({"events_pp": gg["events_pp"], "X_pp": gg["X_pp"], "q_bin": gg["q_bin"][0]}, ref,
                tallies=("q_bin",))


def test_fp64_transient_gaussian_box():
    wl = W.transient_box_c3(n=3000, grid=(16, 16, 8), n_times=20)
    mat, g, run = wl.material, wl.geometries[0], wl.run
    gg = gpu_transient(mat, g, run, L.FP64_PLAIN, per_particle=True)
    ref = oracle.run_transient(mat, g, run, per_particle=True)
    assert np.array_equal(gg["events_pp"], ref["events_pp"])
    ok, err = rel_close(gg["tally"][..., 0], ref["tally"][..., 0], RTOL)
    assert ok, err
    ok, err = rel_close(gg["tally"][..., 1:], ref["tally"][..., 1:], RTOL)
    assert ok, err


def test_fp64_transient_ballistic_walls():
    wl = W.ballistic_transient_e1(n=20_000)
    mat, g, run = wl.material, wl.geometries[0], wl.run
    gg = gpu_transient(mat, g, run, L.FP64_PLAIN, per_particle=True)
    ref = oracle.run_transient(mat, g, run, per_particle=True)
    assert np.array_equal(gg["events_pp"], ref["events_pp"])
    ok, err = rel_close(gg["tally"], ref["tally"], RTOL)
    assert ok, err


def test_fp64_gradient_matches_oracle_scores():
    wl = W.pore_film_c5(n=4000, p_pore=0.3)
    mat, g, run = wl.material, wl.geometries[0], wl.run
    run.max_events = 2_000_000
    rng = np.random.default_rng(5)
    dirs = np.vstack([rng.normal(size=mat.n_bins), np.eye(mat.n_bins)[2500]])
    M = api.Material(mat)
    G = api.Geometry(g)
    cfg = api.SteadyConfig(seed=run.seed, precision=L.FP64_PLAIN, n_scat_max=run.n_scat_max,
                           max_events=run.max_events, tally_axis=run.tally_axis, per_bin=True)
    fwd, go = api.grad(M, G, run.n, cfg, dirs=dirs)
    torch.cuda.synchronize()
    ref = oracle.run_steady(mat, g, run, grad=True, dirs=dirs)
    ok, err = rel_close(go.dkappa_dlogtau.cpu().numpy(), ref["dkappa_dlogtau"], RTOL)
    assert ok, err
    assert go.dkappa_dp[0].item() == pytest.approx(ref["dkappa_dp"], rel=1e-9)
    ok, err = rel_close(go.dkappa_dir[:2, 0].cpu().numpy(), ref["dkappa_dir"], RTOL)
    assert ok, err
    assert fwd.stats[0, L.STAT_KAPPA].item() == pytest.approx(ref["kappa"], rel=RTOL)


def test_edge_single_particle_and_ragged_grid():
    wl = W.gray_slab_c1(n=1)
    mat, g, run = wl.material, wl.geometries[0], wl.run
    for n in (1, 31, 257):
        run.n = n
        gg = gpu_steady(mat, [g], [n], run, L.FP64_PLAIN, per_particle=True)
        ref = oracle.run_steady(mat, g, run, per_particle=True)
        _check_fp64({"events_pp": gg["events_pp"], "X_pp": gg["X_pp"], "T": gg["T"][0], "q": gg["q"][0]}, ref)
        g32 = gpu_steady(mat, [g], [n], run, L.FP32_TRACE, per_particle=True)
        assert g32["stats"][0][L.STAT_N] == n


def test_max_events_truncation_reported():
    wl = W.film_batch_c4(n_films=1)
    mat, g, run = wl.material, wl.geometries[0], wl.run
    run.max_events = 50
    gg = gpu_steady(mat, [g], [2000], run, L.FP64_PLAIN, per_particle=True)
    ref = oracle.run_steady(mat, g, run, n_total=2000, per_particle=True)
    assert gg["stats"][0][L.STAT_STATUS] == L.WARN_TRUNCATED
    assert gg["stats"][0][L.STAT_TRUNCATED] == ref["truncated"] > 0
    assert np.array_equal(gg["events_pp"], ref["events_pp"])
    assert gg["events_pp"].max() == 50


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_time_budget_stops_the_run_and_leaves_the_device_usable(precision):
    # the budget is a device-timer check between events, not a wait: a run
    # that exceeds it stops refilling, reports TIMEOUT, and the next run works
    prec = L.FP32_TRACE if precision == "fp32" else L.FP64_PLAIN
    wl = W.si_slab_c2(n=4_000_000)
    mat, g, run = wl.material, wl.geometries[0], wl.run
    M, G = api.Material(mat), api.Geometry(g)
    cfg = api.SteadyConfig(seed=5, precision=prec, n_cells=run.n_cells, tally_axis=run.tally_axis,
                           time_budget_s=2e-5)
    out = api.run_steady(M, [G], [run.n], cfg)
    torch.cuda.synchronize()
    st = out.stats[0].cpu().numpy()
    assert st[L.STAT_STATUS] == L.ERR_TIMEOUT
    assert st[L.STAT_N] < run.n
    with pytest.raises(L.MCBTEError) as e:           # host outputs: the status comes back as an error
        api.run_steady_host(M, [G], [run.n], cfg)
    assert e.value.status == L.ERR_TIMEOUT
    ok = api.run_steady(M, [G], [20_000], replace(cfg, time_budget_s=0.0))
    torch.cuda.synchronize()
    assert ok.stats[0, L.STAT_STATUS].item() == 0 and ok.stats[0, L.STAT_N].item() == 20_000


def test_host_output_path_matches_device_path():
    wl = W.gray_slab_c1(n=20_000)
    mat, g, run = wl.material, wl.geometries[0], wl.run
    M = api.Material(mat)
    G = api.Geometry(g)
    cfg = api.SteadyConfig(seed=run.seed, precision=L.FP64_PLAIN, n_cells=run.n_cells, tally_axis=2)
    h = api.run_steady_host(M, [G], [run.n], cfg)
    d = api.run_steady(M, [G], [run.n], cfg)
    torch.cuda.synchronize()
    assert rel_close(h["T"], d.T.cpu().numpy(), 1e-12)[0]
    assert h["stats"][0][L.STAT_EVENTS] == d.stats[0, L.STAT_EVENTS].item()


# ------------------------------------------------------------------ FP32 statistical parity
def test_fp32_gray_slab_tallies_within_3se():
    """Cell tallies at the workload's size (1e5 particles per run); kappa on
    larger runs so that 3 combined standard errors are below 0.5 % and both
    bounds of the FP32 contract bind."""
    wl = W.gray_slab_c1()
    mat, g, run = wl.material, wl.geometries[0], wl.run
    M = api.Material(mat)
    gT, gq, gk = [], [], []
    for s in range(8):
        r = gpu_steady(mat, [g], [run.n], run, L.FP32_TRACE, seed=100 + s, M=M)
        gT.append(r["T"][0]); gq.append(r["q"][0][:, 2]); gk.append(r["stats"][0][L.STAT_KAPPA])
    oT, oq, ok_ = [], [], []
    for s in range(8):
        run.seed = 200 + s
        r = oracle.run_steady(mat, g, run)
        oT.append(r["T"]); oq.append(r["q"][:, 2]); ok_.append(r["kappa"])
    for a, b in ((gT, oT), (gq, oq)):
        m1, s1 = batch_stats(a)
        m2, s2 = batch_stats(b)
        z = z_scores(m1, s1, m2, s2)
        assert np.max(np.abs(z)) < 4.0
        assert np.mean(z ** 2) < 2.0
    gk, ok_ = [], []
    for s in range(8):
        gk.append(gpu_steady(mat, [g], [2_000_000], run, L.FP32_TRACE, seed=150 + s, M=M)["stats"][0][L.STAT_KAPPA])
    big = W.SteadyRun(n=500_000, seed=0, n_cells=0, cell_axis=2, tally_axis=2)
    for s in range(8):
        big.seed = 250 + s
        ok_.append(oracle.run_steady(mat, g, big)["kappa"])
    m1, s1 = batch_stats(gk)
    m2, s2 = batch_stats(ok_)
    se = np.hypot(s1, s2)
    assert 3 * se < 0.005 * m2
    assert abs(m1 - m2) < 3 * se and abs(m1 - m2) < 0.005 * m2, (m1, m2, se)


def test_fp32_bvk_slab_kappa_and_spectrum():
    wl = W.si_slab_c2(n=200_000)
    mat, g, run = wl.material, wl.geometries[0], wl.run
    M = api.Material(mat)
    gk, gs, gsp = [], [], []
    for s in range(6):
        r = gpu_steady(mat, [g], [run.n], run, L.FP32_TRACE, seed=300 + s, M=M)
        gk.append(r["stats"][0][L.STAT_KAPPA]); gsp.append(r["q_bin"][0].reshape(30, 100).sum(axis=1))
    ok_, osp = [], []
    for s in range(6):
        run.seed = 400 + s
        r = oracle.run_steady(mat, g, run)
        ok_.append(r["kappa"]); osp.append(r["q_bin"].reshape(30, 100).sum(axis=1))
    m1, s1 = batch_stats(gk)
    m2, s2 = batch_stats(ok_)
    assert abs(m1 - m2) < 3 * np.hypot(s1, s2), (m1, m2, s1, s2)
    z = z_scores(*batch_stats(gsp), *batch_stats(osp))
    assert np.max(np.abs(z)) < 4.0 and np.mean(z ** 2) < 2.5


def test_fp32_film_batch_kappa_vs_oracle():
    wl = W.film_batch_c4(scale=0.02)
    mat, run = wl.material, wl.run
    run.max_events = 20_000_000
    ns = wl.n_per_geom
    gk = []
    M = api.Material(mat)
    r = gpu_steady(mat, wl.geometries, ns, run, L.FP32_TRACE, seed=500, M=M)
    k = r["stats"][:, L.STAT_KAPPA]
    se = r["stats"][:, L.STAT_KAPPA_SE]
    zs = []
    for f in range(0, 64, 9):
        ref = oracle.run_steady(mat, wl.geometries[f], run, n_total=ns[f], batch_index=f)
        run_seed = run.seed
        zs.append((k[f] - ref["kappa"]) / np.hypot(se[f], ref["kappa_se"]))
    zs = np.array(zs)
    assert np.max(np.abs(zs)) < 4.0, zs


def test_fp32_pore_lattice_kappa():
    wl = W.pore_film_c5(n=100_000)
    mat, g, run = wl.material, wl.geometries[0], wl.run
    run.max_events = 20_000_000
    r = gpu_steady(mat, [g], [run.n], run, L.FP32_TRACE, seed=600)
    run.seed = 601
    ref = oracle.run_steady(mat, g, run)
    st = r["stats"][0]
    assert abs(st[L.STAT_KAPPA] - ref["kappa"]) < 3 * np.hypot(st[L.STAT_KAPPA_SE], ref["kappa_se"])


def test_fp32_transient_energy_and_profile():
    wl = W.transient_box_c3(n=200_000, grid=(8, 8, 4), n_times=10)
    mat, g, run = wl.material, wl.geometries[0], wl.run
    r = gpu_transient(mat, g, run, L.FP32_TRACE, seed=700)
    st = r["stats"]
    tb = oracle.tables(mat)
    Vc = 2e-6 * 2e-6 * 1e-6 / (8 * 8 * 4)
    tot = r["tally"][..., 0].sum(axis=(1, 2, 3)) * tb["C_tot"] * Vc
    assert np.allclose(tot, st[L.STAT_E_TOT], rtol=1e-12)
    # z-profile (summed over x, y) against the oracle on independent streams:
    # 16 oracle batches (disjoint particle ranges of another seed), 8 GPU seeds
    orun = W.transient_box_c3(n=400_000, grid=(8, 8, 4), n_times=10).run
    orun.seed = 710
    vals = []
    nb = 16
    for b in range(nb):
        a, e = orun.n * b // nb, orun.n * (b + 1) // nb
        rr = oracle.run_transient(mat, g, orun, pid_begin=a, pid_end=e)
        vals.append(rr["tally"][..., 0].sum(axis=(2, 3)) * (orun.n / (e - a)))
    m2, s2 = batch_stats(vals)
    gvals = []
    for s in range(8):
        gvals.append(gpu_transient(mat, g, run, L.FP32_TRACE, seed=720 + s)["tally"][..., 0].sum(axis=(2, 3)))
    m1, s1 = batch_stats(gvals)
    z = z_scores(m1, s1, m2, s2)
    assert np.max(np.abs(z)) < 5.0 and np.mean(z ** 2) < 2.5, z


def test_fp32_ballistic_transient_analytic():
    from oracle import closed_forms as cf
    wl = W.ballistic_transient_e1(n=2_000_000, nz=30)
    mat, g, run = wl.material, wl.geometries[0], wl.run
    r = gpu_transient(mat, g, run, L.FP32_TRACE)
    T = r["tally"][:, :, 0, 0, 0]
    L_ = 3e-6
    for m, t in enumerate(run.t_meas):
        fine = np.linspace(0, L_, 30 * 50 + 1)
        ex = cf.ballistic_transient(fine, t, L_, 12360.0, 3.0, -3.0)
        exc = np.array([ex[i * 50:(i + 1) * 50 + 1].mean() for i in range(30)])
        assert np.max(np.abs(T[m] - exc)) < 0.06, (t, np.max(np.abs(T[m] - exc)))


def test_fp32_gradient_directional_vs_oracle():
    wl = W.pore_film_c5(n=100_000, p_pore=0.3)
    mat, g, run = wl.material, wl.geometries[0], wl.run
    run.max_events = 20_000_000
    rng = np.random.default_rng(9)
    dirs = np.vstack([rng.choice([-1.0, 1.0], size=mat.n_bins), np.eye(mat.n_bins)[100]])
    M = api.Material(mat)
    G = api.Geometry(g)
    cfg = api.SteadyConfig(seed=800, precision=L.FP32_TRACE, n_scat_max=run.n_scat_max,
                           max_events=run.max_events, tally_axis=run.tally_axis, per_bin=True)
    fwd, go = api.grad(M, G, run.n, cfg, dirs=dirs)
    torch.cuda.synchronize()
    assert fwd.stats[0, L.STAT_STATUS].item() == 0      # no replay mismatch, no truncation
    run.seed = 801
    ref = oracle.run_steady(mat, g, run, grad=True, dirs=dirs)
    gd = go.dkappa_dir[:2].cpu().numpy()
    for k in range(2):
        se = np.hypot(gd[k, 1], ref["dkappa_dir_se"][k])
        assert abs(gd[k, 0] - ref["dkappa_dir"][k]) < 4 * se
    gp = go.dkappa_dp.cpu().numpy()
    assert abs(gp[0] - ref["dkappa_dp"]) < 4 * np.hypot(gp[1], ref["dkappa_dp_se"])


@pytest.mark.parametrize("p_pore,est", [(0.0, L.DP_AUTO), (0.3, L.DP_MEASURE_VALUED), (1.0, L.DP_AUTO)])
def test_fp64_measure_valued_specularity_gradient_matches_oracle(p_pore, est):
    wl = W.pore_film_c5(n=4000, p_pore=p_pore)
    mat, g, run = wl.material, wl.geometries[0], wl.run
    run.max_events = 2_000_000
    M, G = api.Material(mat), api.Geometry(g)
    cfg = api.SteadyConfig(seed=run.seed, precision=L.FP64_PLAIN, n_scat_max=run.n_scat_max,
                           max_events=run.max_events, tally_axis=run.tally_axis, per_bin=True)
    fwd, go = api.grad(M, G, run.n, cfg, dp_estimator=est)
    torch.cuda.synchronize()
    ref = oracle.run_steady(mat, g, run, grad=True, dp_estimator=est)
    dp = go.dkappa_dp.cpu().numpy()
    assert dp[0] == pytest.approx(ref["dkappa_dp"], rel=1e-9)
    assert dp[1] == pytest.approx(ref["dkappa_dp_se"], rel=1e-9)
    # the phantom traces change neither the forward tallies nor the tau gradient
    ok, err = rel_close(go.dkappa_dlogtau.cpu().numpy(), ref["dkappa_dlogtau"], RTOL)
    assert ok, err
    assert fwd.stats[0, L.STAT_KAPPA].item() == pytest.approx(ref["kappa"], rel=RTOL)
    assert fwd.stats[0, L.STAT_EVENTS].item() == ref["events"]
    if p_pore in (0.0, 1.0):
        # the likelihood ratio is undefined there: NaN on request
        _, gl = api.grad(M, G, run.n, cfg, dp_estimator=L.DP_LIKELIHOOD_RATIO)
        torch.cuda.synchronize()
        assert np.isnan(gl.dkappa_dp.cpu().numpy()).all()


def test_fp32_measure_valued_specularity_gradient_vs_oracle():
    wl = W.pore_film_c5(n=100_000, p_pore=0.0)
    mat, g, run = wl.material, wl.geometries[0], wl.run
    run.max_events = 20_000_000
    M, G = api.Material(mat), api.Geometry(g)
    cfg = api.SteadyConfig(seed=810, precision=L.FP32_TRACE, n_scat_max=run.n_scat_max,
                           max_events=run.max_events, tally_axis=run.tally_axis, per_bin=True)
    fwd, go = api.grad(M, G, run.n, cfg)
    torch.cuda.synchronize()
    assert fwd.stats[0, L.STAT_STATUS].item() == 0      # no replay mismatch, no truncation
    run.seed = 811
    ref = oracle.run_steady(mat, g, run, grad=True)     # measure-valued at p = 0
    gp = go.dkappa_dp.cpu().numpy()
    assert np.isfinite(gp).all() and gp[1] > 0
    assert abs(gp[0] - ref["dkappa_dp"]) < 4 * np.hypot(gp[1], ref["dkappa_dp_se"])


def test_grad_rejects_unknown_dp_estimator():
    wl = W.pore_film_c5(n=100)
    M, G = api.Material(wl.material), api.Geometry(wl.geometries[0])
    cfg = api.SteadyConfig(seed=1, precision=L.FP64_PLAIN, n_scat_max=4, tally_axis=1)
    with pytest.raises(L.MCBTEError) as e:
        api.grad(M, G, 100, cfg, dp_estimator=3)
    assert e.value.status == L.ERR_INVALID_ARG


def test_nscat_curve_fp64_matches_oracle_and_fp32_statistics():
    # kappa for every N_scat_max from one run (Sec. 3.5.6), off-centre pore
    # with a diagonal control gradient
    m = W.bvk_holland(n_per_branch=50)
    g = W.pore_skew()
    run = W.SteadyRun(n=20_000, seed=62, tally_axis=1, n_scat_max=16, max_events=10 ** 7)
    ref = oracle.run_steady(m, g, run, nscat_curve=True)
    M, G = api.Material(m), api.Geometry(g)
    base = dict(n_scat_max=run.n_scat_max, max_events=run.max_events, tally_axis=1, nscat_curve=True)
    o = api.run_steady(M, [G], [run.n], api.SteadyConfig(seed=run.seed, precision=L.FP64_PLAIN, **base))
    torch.cuda.synchronize()
    kn = o.kappa_nscat[0].cpu().numpy()
    ok, err = rel_close(kn, ref["kappa_nscat"], 1e-9)
    assert ok, err
    assert kn[-1, 0] == pytest.approx(o.stats[0, L.STAT_KAPPA].item(), rel=1e-12)
    # host outputs through the C ABI: the same curve
    h = api.run_steady_host(M, [G], [run.n], api.SteadyConfig(seed=run.seed, precision=L.FP64_PLAIN, **base))
    ok, err = rel_close(h["kappa_nscat"][0], ref["kappa_nscat"], 1e-9)
    assert ok, err
    # FP32: an independent sample, every point within 4 combined SE; the last
    # point is the run's own kappa, which a plain run reproduces
    n32 = 400_000
    c32 = api.SteadyConfig(seed=63, precision=L.FP32_TRACE, **base)
    o32 = api.run_steady(M, [G], [n32], c32)
    plain = api.run_steady(M, [G], [n32], replace(c32, nscat_curve=False))
    torch.cuda.synchronize()
    k32 = o32.kappa_nscat[0].cpu().numpy()
    assert o32.stats[0, L.STAT_STATUS].item() == 0
    assert o32.stats[0, L.STAT_KAPPA].item() == pytest.approx(plain.stats[0, L.STAT_KAPPA].item(), rel=1e-3)
    assert k32[-1, 0] == pytest.approx(o32.stats[0, L.STAT_KAPPA].item(), rel=1e-9)
    ref2 = oracle.run_steady(m, g, replace(run, n=200_000, seed=64), nscat_curve=True)
    z = (k32[:, 0] - ref2["kappa_nscat"][:, 0]) / np.hypot(k32[:, 1], ref2["kappa_nscat"][:, 1])
    assert np.all(np.abs(z) < 4.0), z


def test_nscat_curve_rejected_with_gradient_and_without_output():
    wl = W.pore_film_c5(n=100)
    M, G = api.Material(wl.material), api.Geometry(wl.geometries[0])
    cfg = api.SteadyConfig(seed=1, precision=L.FP64_PLAIN, n_scat_max=4, tally_axis=1, nscat_curve=True)
    with pytest.raises(L.MCBTEError) as e:
        api.grad(M, G, 100, cfg)
    assert e.value.status == L.ERR_INVALID_ARG
    out = api.SteadyOutputs(1, M.n_bins, 0, False)          # no kappa_nscat buffer
    with pytest.raises(L.MCBTEError) as e:
        api.run_steady(M, [G], [100], cfg, out=out)
    assert e.value.status == L.ERR_INVALID_ARG
    with pytest.raises(L.MCBTEError) as e:
        api.run_steady(M, [G], [100], replace(cfg, n_scat_max=0))
    assert e.value.status == L.ERR_INVALID_ARG


def test_steady_detectors_per_frequency_bin():
    m = W.bvk_holland(n_per_branch=20)
    wl = W.si_slab_c2(n=20_000, material=m)
    g, run = wl.geometries[0], wl.run
    Lb = g.L
    tiles = ((0.0, Lb[0], 0.0, Lb[1], 0.0, Lb[2]), (2, 2, 4))
    sub = ((0.1 * Lb[0], 0.7 * Lb[0], 0.0, Lb[1], 0.25 * Lb[2], 0.75 * Lb[2]), (2, 1, 3))
    run = replace(run, regions=[tiles, sub])
    M, G = api.Material(m), api.Geometry(g)
    base = dict(seed=run.seed, n_cells=run.n_cells, cell_axis=2, tally_axis=2, per_bin=True,
                max_events=run.max_events, regions=run.regions, det_per_bin=True)
    o = api.run_steady(M, [G], [run.n], api.SteadyConfig(precision=L.FP64_PLAIN, **base))
    torch.cuda.synchronize()
    ref = oracle.run_steady(m, g, run, det_per_bin=True)
    d = o.det.cpu().numpy()
    assert d.shape == (22, m.n_bins, 4)
    ok, err = rel_close(d[..., 0], ref["det_T"], RTOL)
    assert ok, err
    ok, err = rel_close(d[..., 1:], ref["det_q"], RTOL)
    assert ok, err
    # host outputs through the C ABI carry the same array
    h = api.run_steady_host(M, [G], [run.n], api.SteadyConfig(precision=L.FP64_PLAIN, **base))
    assert h["stats"][0, L.STAT_KAPPA] == pytest.approx(o.stats[0, L.STAT_KAPPA].item(), rel=1e-12)
    ok, err = rel_close(h["det"], d, RTOL)
    assert ok, err
    # FP32: the bins of each detector sum to the detector total of a run
    # without the split (exact fixed-point sums, same trajectories)
    c32 = api.SteadyConfig(precision=L.FP32_TRACE, **base)
    o32 = api.run_steady(M, [G], [500_000], c32)
    t32 = api.run_steady(M, [G], [500_000], replace(c32, det_per_bin=False))
    torch.cuda.synchronize()
    s = o32.det.sum(dim=1).cpu().numpy()
    t = t32.det.cpu().numpy()
    np.testing.assert_allclose(s, t, rtol=1e-9, atol=1e-12 * np.abs(t).max())
    # and the tiles give back the frequency-resolved flux
    vd = float(np.prod(Lb)) / 16
    q_tiles = (vd * o32.det[:16, :, 3]).sum(dim=0).cpu().numpy() / float(np.prod(Lb))
    qb = o32.q_bin[0].cpu().numpy()
    np.testing.assert_allclose(q_tiles, qb, rtol=1e-6, atol=1e-9 * np.abs(qb).max())


def test_det_per_bin_needs_regions():
    wl = W.si_slab_c2(n=100)
    M, G = api.Material(wl.material), api.Geometry(wl.geometries[0])
    with pytest.raises(L.MCBTEError) as e:
        api.run_steady(M, [G], [100], api.SteadyConfig(seed=1, precision=L.FP64_PLAIN, tally_axis=2, det_per_bin=True))
    assert e.value.status == L.ERR_INVALID_ARG


def test_nscat_curve_per_geometry_in_a_batch():
    # the curve's accumulators are kept per geometry: three films of one
    # batched launch, each against the oracle run of that film alone
    wl = W.film_batch_c4(n_films=3)
    mat, run = wl.material, wl.run
    run.max_events = 2_000_000
    ns = [700, 257, 1000]
    M = api.Material(mat)
    Gs = [api.Geometry(g) for g in wl.geometries]
    cfg = api.SteadyConfig(seed=run.seed, precision=L.FP64_PLAIN, tally_axis=run.tally_axis,
                           n_scat_max=run.n_scat_max, max_events=run.max_events, nscat_curve=True)
    o = api.run_steady(M, Gs, ns, cfg)
    torch.cuda.synchronize()
    kn = o.kappa_nscat.cpu().numpy()
    assert kn.shape == (3, run.n_scat_max, 2)
    for f in range(3):
        ref = oracle.run_steady(mat, wl.geometries[f], run, n_total=ns[f], batch_index=f, nscat_curve=True)
        ok, err = rel_close(kn[f], ref["kappa_nscat"], RTOL)
        assert ok, (f, err)


def test_nscat_curve_4096_points_matches_a_short_run():
    # the longest curve (its sums kept in fewer copies than a short curve's):
    # on the same trajectories, the point at k = 16 is the kappa of a run with
    # N_scat_max = 16, and the last point the run's own kappa
    m = W.bvk_holland(n_per_branch=20)
    wl = W.si_slab_c2(n=300_000, material=m)
    M, G = api.Material(m), api.Geometry(wl.geometries[0])
    c = api.SteadyConfig(seed=71, precision=L.FP32_TRACE, tally_axis=2, n_scat_max=4096, nscat_curve=True,
                         max_events=10 ** 7)
    o = api.run_steady(M, [G], [wl.run.n], c)
    s16 = api.run_steady(M, [G], [wl.run.n], replace(c, n_scat_max=16, nscat_curve=False))
    torch.cuda.synchronize()
    kn = o.kappa_nscat[0].cpu().numpy()
    assert kn.shape == (4096, 2)
    assert o.stats[0, L.STAT_STATUS].item() == 0 and s16.stats[0, L.STAT_STATUS].item() == 0
    assert kn[-1, 0] == pytest.approx(o.stats[0, L.STAT_KAPPA].item(), rel=1e-9)
    assert kn[15, 0] == pytest.approx(s16.stats[0, L.STAT_KAPPA].item(), rel=1e-9)
    assert kn[15, 1] == pytest.approx(s16.stats[0, L.STAT_KAPPA_SE].item(), rel=1e-6)


def test_fp32_measure_valued_specularity_gradient_at_p1():
    wl = W.pore_film_c5(n=100_000, p_pore=1.0)
    mat, g, run = wl.material, wl.geometries[0], wl.run
    run.max_events = 20_000_000
    M, G = api.Material(mat), api.Geometry(g)
    cfg = api.SteadyConfig(seed=820, precision=L.FP32_TRACE, n_scat_max=run.n_scat_max,
                           max_events=run.max_events, tally_axis=run.tally_axis, per_bin=True)
    fwd, go = api.grad(M, G, run.n, cfg)
    torch.cuda.synchronize()
    assert fwd.stats[0, L.STAT_STATUS].item() == 0
    run.seed = 821
    ref = oracle.run_steady(mat, g, run, grad=True)     # measure-valued at p = 1
    gp = go.dkappa_dp.cpu().numpy()
    assert np.isfinite(gp).all() and gp[1] > 0
    assert abs(gp[0] - ref["dkappa_dp"]) < 4 * np.hypot(gp[1], ref["dkappa_dp_se"])


def test_large_tables_global_memory_paths():
    # 12 000 bins: the alias build works in global scratch (beyond its
    # shared-memory size), the FP32 tracer keeps the per-bin constants out
    # of shared memory; tables bit-identical, FP64 run identical per
    # particle, FP32 kappa within the combined standard error
    rng = np.random.default_rng(12)
    n = 12_000
    m = W.Material(omega=np.linspace(1e12, 7e13, n), v=rng.uniform(1e3, 9e3, n), tau=10 ** rng.uniform(-12, -10, n),
                   C=rng.exponential(size=n) * 1e3, T_lin=300.0)
    M = api.Material(m)
    t_g, t_o = M.tables(), oracle.tables(m)
    for k in ("C", "alias", "thr", "prob"):
        assert np.array_equal(t_g[k], t_o[k]), k
    wl = W.gray_slab_c1(n=3000)
    g, run = wl.geometries[0], wl.run
    run.n_cells = 10
    gg = gpu_steady(m, [g], [run.n], run, L.FP64_PLAIN, per_particle=True)
    ref = oracle.run_steady(m, g, run, per_particle=True)
    _check_fp64({"events_pp": gg["events_pp"], "X_pp": gg["X_pp"], "T": gg["T"][0], "q": gg["q"][0]}, ref)
    G = api.Geometry(g)
    o32 = api.run_steady(M, [G], [200_000], api.SteadyConfig(seed=77, precision=L.FP32_TRACE, n_cells=10,
                                                             cell_axis=2, tally_axis=2, per_bin=True))
    torch.cuda.synchronize()
    s32 = o32.stats[0].cpu().numpy()
    assert s32[L.STAT_STATUS] == 0
    ref2 = oracle.run_steady(m, g, replace(run, n=200_000, seed=78))
    assert abs(s32[L.STAT_KAPPA] - ref2["kappa"]) < 4 * np.hypot(s32[L.STAT_KAPPA_SE], ref2["kappa_se"])


def test_fp32_two_block_relaxation_draw_beyond_65536_bins():
    # more bins than the one-block FP32 relaxation draw serves: the FP32
    # tracer takes the two-block draw of the FP64 path (64-bit threshold)
    rng = np.random.default_rng(13)
    n = 70_000
    m = W.Material(omega=np.linspace(1e12, 7e13, n), v=rng.uniform(1e3, 9e3, n), tau=10 ** rng.uniform(-12, -10, n),
                   C=rng.exponential(size=n) * 1e3, T_lin=300.0)
    M = api.Material(m)
    wl = W.gray_slab_c1(n=2000)
    g, run = wl.geometries[0], wl.run
    run.n_cells = 10
    gg = gpu_steady(m, [g], [run.n], run, L.FP64_PLAIN, per_particle=True, M=M)
    ref = oracle.run_steady(m, g, run, per_particle=True)
    _check_fp64({"events_pp": gg["events_pp"], "X_pp": gg["X_pp"], "T": gg["T"][0], "q": gg["q"][0]}, ref)
    G = api.Geometry(g)
    o32 = api.run_steady(M, [G], [200_000], api.SteadyConfig(seed=79, precision=L.FP32_TRACE, n_cells=10,
                                                             cell_axis=2, tally_axis=2))
    torch.cuda.synchronize()
    s32 = o32.stats[0].cpu().numpy()
    assert s32[L.STAT_STATUS] == 0
    ref2 = oracle.run_steady(m, g, replace(run, n=200_000, seed=80))
    assert abs(s32[L.STAT_KAPPA] - ref2["kappa"]) < 4 * np.hypot(s32[L.STAT_KAPPA_SE], ref2["kappa_se"])
