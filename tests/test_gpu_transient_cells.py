"""FP32 transient tallies cell by cell and time by time against the oracle.

The hot-spot box of the transient workload (2 x 2 x 1 um, diffuse adiabatic
walls, +1 K Gaussian of sigma 100 nm at the top-face centre) on its full
64 x 64 x 32 grid, at six of its measurement times (10, 20, 100, 500, 1000 and
2000 ps; the last is t_max), two times per time window so that particles are
parked and resumed between windows as in a full run.  Both FP32 kernel
variants are covered: snapshots at t_m (Eq. sampling, Sec. 3.4) and averages
over [t_{m-1}, t_m) (Sec. 4.5).

The GPU side is 64 independent runs of 1e6 particles.  Their spread gives the
per-run variance s^2 of every tally entry; under the null hypothesis the
oracle's single run of N_o = 1e6 particles has the same per-particle law, so
its variance is s^2 n_run / N_o.  Every cell, time and component (T, q_x,
q_y, q_z) whose cell holds at least 30 particles on average is compared:
    z = (mean_gpu - oracle) / (s sqrt(1/64 + n_run / N_o)),
which is Student-t with 63 degrees of freedom.  About 1e5 values are
compared; max |z| < 6.5 keeps the family-wise false-alarm rate near 2e-3
(Bonferroni), and the mean of z^2 (63/61 = 1.03 expected, spread about 0.01)
must stay below 1.15, which catches a bias of a third of a standard error
spread over the cells.
"""
import numpy as np
import pytest

import oracle
from inputs import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2104_03573_gb300 import _lib as L  # noqa: E402
from paper_2104_03573_gb300 import api  # noqa: E402

T_MEAS = np.array([10.0, 20.0, 100.0, 500.0, 1000.0, 2000.0]) * 1e-12
N_RUN = 1_000_000
N_RUNS = 64
N_ORACLE = 1_000_000


def _box(time_average):
    wl = W.transient_box_c3(n=N_RUN)
    m, g, run = wl.material, wl.geometries[0], wl.run
    run.t_meas = T_MEAS
    run.t_max = float(T_MEAS[-1])
    run.time_average = time_average
    return m, g, run


@pytest.mark.parametrize("time_average", [False, True])
def test_fp32_transient_every_cell_and_time_vs_oracle(time_average):
    m, g, run = _box(time_average)
    M, G = api.Material(m), api.Geometry(g)
    s1 = s2 = None
    e_tot = None
    for b in range(N_RUNS):
        cfg = api.TransientConfig(seed=91_000 + b, t_max=run.t_max, t_meas=run.t_meas, grid=run.grid,
                                  precision=L.FP32_TRACE, window_times=2, time_average=time_average)
        out = api.run_transient(M, G, N_RUN, cfg)
        x = out.tally
        s1 = x.clone() if s1 is None else s1 + x
        s2 = x * x if s2 is None else s2 + x * x
        assert out.stats[L.STAT_STATUS].item() == 0
        e_tot = out.stats[L.STAT_E_TOT].item()
    torch.cuda.synchronize()
    mean = (s1 / N_RUNS).cpu().numpy()
    var = ((s2 - s1 * s1 / N_RUNS) / (N_RUNS - 1)).clamp_min(0.0).cpu().numpy()
    run.n = N_ORACLE
    run.seed = 97_003
    ref = oracle.run_transient(m, g, run)["tally"]
    # particles per cell and run: T is (E_tot / n) / (C_tot V_cell) per particle
    quantum = (e_tot / N_RUN) / (oracle.tables(m)["C_tot"] * (4e-18 / (64 * 64 * 32)))
    occupied = mean[..., 0] / quantum >= 30.0
    sel = np.broadcast_to(occupied[..., None], mean.shape)
    assert occupied.sum(axis=(1, 2, 3)).min() > 1000          # every time has well-filled cells
    sd = np.sqrt(var[sel] * (1.0 / N_RUNS + N_RUN / N_ORACLE))
    assert np.all(sd > 0)
    z = (mean[sel] - ref[sel]) / sd
    zc = z.reshape(-1, 4)
    msg = f"{z.size} values, max|z| {np.abs(z).max():.2f}, mean z^2 per component {np.mean(zc ** 2, axis=0)}"
    assert np.abs(z).max() < 6.5, msg
    assert np.mean(z ** 2) < 1.15, msg
    for k in range(4):                                          # T, q_x, q_y, q_z separately
        assert np.mean(zc[:, k] ** 2) < 1.2, msg
