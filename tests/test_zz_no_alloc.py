"""The allocation-free steady run, for callers that cannot allocate device
memory, must give the same results as the regular steady run.

``mcbte_run_steady_noalloc`` keeps its scratch in a fixed device array
inside the library instead of a caller workspace or cudaMallocAsync.  It is
called here twice in a row through the C ABI: the second call reuses the
array left behind by the first, so it also checks that everything that must
start at zero is cleared on each call, and that the second call leaves the
device's free memory unchanged (the first may still load device code).  The
tolerance is the one the other parity tests use (1e-9 of the tally's largest
magnitude; per-particle event counts and X_p identical).  This file is
collected last on purpose.
"""
import numpy as np
import pytest

from inputs import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2104_03573_gb300 import _lib as L  # noqa: E402
from paper_2104_03573_gb300 import api  # noqa: E402

RTOL = 1e-9


def _close(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.max(np.abs(a - b)) <= RTOL * max(np.max(np.abs(b)), 1e-300)


@pytest.mark.parametrize("precision", [L.FP64_PLAIN, L.FP32_TRACE])
def test_noalloc_matches_regular_steady_run_twice(precision):
    wl = W.si_slab_c2(n=30_000)
    mat, geo, run = wl.material, wl.geometries[0], wl.run
    M = api.Material(mat)
    G = api.Geometry(geo)
    cfg = api.SteadyConfig(seed=run.seed, precision=precision, n_cells=run.n_cells, cell_axis=2, tally_axis=2,
                           per_bin=True)
    ref = api.run_steady(M, [G], [run.n], cfg, per_particle=True)
    torch.cuda.synchronize()
    for call in range(2):
        out = api.SteadyOutputs(1, M.n_bins, run.n_cells, True, run.n, per_particle=True)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        api.run_steady_noalloc(M, [G], [run.n], cfg, out)
        torch.cuda.synchronize()
        if call == 1:
            assert torch.cuda.mem_get_info()[0] == free_before
        assert torch.equal(out.events_pp, ref.events_pp)
        assert torch.equal(out.X_pp, ref.X_pp)
        assert _close(out.T.cpu().numpy(), ref.T.cpu().numpy())
        assert _close(out.q.cpu().numpy(), ref.q.cpu().numpy())
        assert _close(out.q_bin.cpu().numpy(), ref.q_bin.cpu().numpy())
        s, r = out.stats[0].cpu().numpy(), ref.stats[0].cpu().numpy()
        assert s[L.STAT_EVENTS] == r[L.STAT_EVENTS]
        assert s[L.STAT_N] == r[L.STAT_N] == run.n
        assert abs(s[L.STAT_KAPPA] - r[L.STAT_KAPPA]) <= RTOL * abs(r[L.STAT_KAPPA])


def test_noalloc_rejects_runs_beyond_its_scratch():
    n_bins = 200_000
    rng = np.random.default_rng(0)
    mat = W.Material(omega=np.linspace(1e11, 7e13, n_bins), v=rng.uniform(1e3, 9e3, n_bins),
                     tau=np.full(n_bins, 1e-11), C=np.ones(n_bins), T_lin=300.0)
    M = api.Material(mat)
    geoms = [api.Geometry(W.film(50e-9)) for _ in range(8)]    # 8 x 200k per-bin accumulators > 8 MiB
    cfg = api.SteadyConfig(seed=1, precision=L.FP32_TRACE, tally_axis=1, per_bin=True, n_scat_max=2)
    out = api.SteadyOutputs(8, n_bins, 0, True)
    with pytest.raises(L.MCBTEError) as e:
        api.run_steady_noalloc(M, geoms, [100] * 8, cfg, out)
    assert e.value.status == L.ERR_WORKSPACE
    assert "scratch" in str(e.value)
    o = L.SteadyOut()
    o.on_host = 1
    assert L.load().mcbte_run_steady_noalloc(M.handle, api._handles(geoms), 1, None, o, None) == L.ERR_INVALID_ARG
