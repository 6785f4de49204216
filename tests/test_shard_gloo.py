"""Multi-rank path on CPU: two gloo ranks each trace a contiguous range of
one run's particles under the run's single key (the oracle stands in for
the GPU tracer), then the shard module sums the tallies and pools the
statistics.  The result is the single-process run of all the particles:
per-particle event counts and X_p bit for bit, tallies and kappa to the
rounding of a different summation order, standard errors from the pooled
sums."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

pytest.importorskip("torch")

import oracle  # noqa: E402
from inputs import workloads as W  # noqa: E402
from paper_2104_03573_gb300 import _lib as L, shard  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shard_ranges_cover_the_run():
    for n, world in ((10, 3), (1_000_003, 8), (5, 8)):
        ranges = [shard.shard_range(n, r, world) for r in range(world)]
        assert sum(c for _, c in ranges) == n
        assert all(ranges[r][0] + ranges[r][1] == ranges[r + 1][0] for r in range(world - 1))


def test_rank_keys_are_distinct():
    assert len({shard.rank_key(1001, r) for r in range(64)}) == 64


def test_two_gloo_ranks_equal_the_single_run(tmp_path):
    n = 30_001
    port = _free_port()
    env = dict(os.environ, MASTER_ADDR="127.0.0.1", GLOO_SOCKET_IFNAME=os.environ.get("GLOO_SOCKET_IFNAME", "lo"))
    procs = [subprocess.Popen([sys.executable, os.path.join(HERE, "shard_worker.py"), str(r), "2", str(port),
                               str(tmp_path), str(n)], env=env) for r in range(2)]
    assert [p.wait(timeout=300) for p in procs] == [0, 0]
    got = json.loads((tmp_path / "rank0.json").read_text())
    pooled = np.array(got["stats"])
    tall = np.load(tmp_path / "tallies.npy")
    pp = np.concatenate([np.load(tmp_path / f"pp{r}.npy") for r in range(2)], axis=1)

    wl = W.si_slab_c2(n=n, material=W.bvk_holland(n_per_branch=20))
    ref = oracle.run_steady(wl.material, wl.geometries[0], wl.run, per_particle=True, n_threads=2)
    assert np.array_equal(pp[0], ref["events_pp"].astype(np.float64))
    assert np.array_equal(pp[1].view(np.int64), ref["X_pp"].view(np.int64))
    want = np.concatenate([ref["T"].ravel(), ref["q"].ravel(), ref["q_bin"].ravel()])
    np.testing.assert_allclose(tall, want, rtol=1e-12, atol=1e-12 * np.abs(want).max())
    assert pooled[L.STAT_N] == n and pooled[L.STAT_EVENTS] == ref["events"]
    assert pooled[L.STAT_KAPPA] == pytest.approx(ref["kappa"], rel=1e-12)
    assert pooled[L.STAT_Q_MEAN] == pytest.approx(ref["q_mean"], rel=1e-12)
    assert pooled[L.STAT_KAPPA_SE] == pytest.approx(ref["kappa_se"], rel=1e-9)
    assert pooled[L.STAT_SIGNED_ABSORBED] == pooled[L.STAT_SIGNED_EMITTED]
    assert got["t_max"] == 2.0
