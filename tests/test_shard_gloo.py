"""Multi-rank path on CPU: two gloo ranks, each tracing its own independent
sample (the oracle stands in for the GPU tracer), pool the kappa estimator's
accumulators and take the maximum of their timings."""
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


def _row(r, n):
    row = np.zeros(L.NSTATS)
    row[L.STAT_N] = n
    row[L.STAT_SUMX] = r["scal"][oracle.SUMX]
    row[L.STAT_SUMX2] = r["scal"][oracle.SUMX2]
    row[L.STAT_EVENTS] = r["events"]
    row[L.STAT_KAPPA] = r["kappa"]
    return row


def test_rank_keys_are_distinct():
    keys = {shard.rank_key(1001, r) for r in range(64)}
    assert len(keys) == 64


def test_two_gloo_ranks_pool_the_estimator(tmp_path):
    n = 20_000
    port = _free_port()
    out = tmp_path / "rank0.json"
    env = dict(os.environ, MASTER_ADDR="127.0.0.1", GLOO_SOCKET_IFNAME=os.environ.get("GLOO_SOCKET_IFNAME", "lo"))
    procs = [subprocess.Popen([sys.executable, os.path.join(HERE, "shard_worker.py"), str(r), "2", str(port), str(out),
                               str(n)], env=env) for r in range(2)]
    rcs = [p.wait(timeout=300) for p in procs]
    assert rcs == [0, 0]
    got = json.loads(out.read_text())

    # the same two samples pooled in one process
    wl = W.gray_slab_c1(n=n)
    rows, ks = [], []
    for r in range(2):
        run = wl.run
        run.seed = shard.rank_key(1001, r)
        res = oracle.run_steady(wl.material, wl.geometries[0], run, n_threads=2)
        rows.append(_row(res, n))
        ks.append(res["kappa"])
    ref = shard.combine_steady_stats(rows)
    for k in ("n", "events", "kappa", "kappa_se"):
        assert got["pooled"][k] == pytest.approx(ref[k], rel=1e-12, abs=0), k
    assert got["pooled"]["n"] == 2 * n
    assert got["events"] == pytest.approx(rows[0][L.STAT_EVENTS] + rows[1][L.STAT_EVENTS], rel=0, abs=0)
    assert got["t_max"] == 2.0
    # the pooled estimate is the particle-weighted mean of the ranks' estimates,
    # with a standard error about 1/sqrt(2) of one rank's
    assert ref["kappa"] == pytest.approx(0.5 * (ks[0] + ks[1]), rel=1e-12)
    se1 = [shard.combine_steady_stats([r])["kappa_se"] for r in rows]
    assert ref["kappa_se"] == pytest.approx(np.mean(se1) / np.sqrt(2), rel=0.05)
