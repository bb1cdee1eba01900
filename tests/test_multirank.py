"""The N > 1 path of bench.py on CPU: world-size-2 gloo process groups.

The bench runs the single-graph workloads as one independent replica per
GPU, splits the batch's graphs and the served job stream over the ranks, and
exchanges only the whole-job figures after the timed region: the slowest
rank's time (MAX) and the sum of the ranks' pair-updates (SUM).  Under
torchrun the reference arm runs on rank 0 only; other ranks exit 0 without
work.  One graph split over vertex-range shards runs the product's exchange
over gloo on an oracle-backed engine, also with one rank failing.
"""
import json
import multiprocessing as mp
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_combine_ranks_gloo_world_2():
    import _rank_worker
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_worker.combine, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        res = sorted(q.get(timeout=120) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs)
    for rank, t, pairs, v, none in res:
        assert t == 2.0            # slowest rank
        assert pairs == 300.0      # 100 + 200
        assert v == 6.0            # 2 + 4
        assert none is None


def test_job_shares_gloo_world_2():
    """The batched and served forms split their independent jobs over the
    ranks: computed on each rank alone, the shares agree, are disjoint and
    cover every graph and every job of the stream; the graph shares carry
    nearly equal work."""
    import _rank_worker
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_worker.shares, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        res = sorted(q.get(timeout=120) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs)
    (_, got0, sizes), (_, got1, _) = res
    assert got0 == got1
    (g0, j0), (g1, j1) = got0
    assert sorted(g0 + g1) == list(range(256)) and not set(g0) & set(g1)
    assert sorted(j0 + j1) == list(range(200)) and not set(j0) & set(j1)
    w0, w1 = sum(sizes[i] for i in g0), sum(sizes[i] for i in g1)
    assert abs(w0 - w1) <= max(sizes)


def test_combine_ranks_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks(1.5, 10) == (1.5, 10.0)
    assert bench.sum_ranks(3.0) == 3.0


@pytest.mark.parametrize("rank", [0, 1])
def test_reference_arm_rank_zero_only(rank):
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], env=env, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    if rank == 0:
        assert len(lines) == 1
        line = json.loads(lines[0])
        assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
        assert line["cpu_baseline"]["kind"] == "oracle"
        assert line["e2e"]["h2d_bytes_per_step"] == 0
    else:
        assert lines == []


@pytest.mark.parametrize("form", ["per-vertex", "block"])
def test_sharded_graph_gloo_world_2(form):
    """One graph over two ranks (Sec. III.E's split of Eq. 3's sums): each
    rank evaluates its vertex range, the product's exchange (ShardRank:
    all-reduce of the sums and histograms, gather of the positions) runs over
    gloo, and after two epochs both ranks hold the positions and sigma of the
    oracle's whole-graph run (up to the order of FP64 additions)."""
    import _rank_worker
    import numpy as np
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2011_03479_gb300 import inputs
    oracle.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_worker.shard_epochs, args=(r, 2, port, q, form)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        res = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs)
    w = inputs.sbm_1000()
    rp, ci = w["row_ptr"], w["col_idx"]
    d, k, kw = (2, 5, {}) if form == "per-vertex" else (16, 0, {"block_partners": 64})
    x0 = oracle.init_positions(1000, d, 99).astype(np.float64)
    xr, sr, _ = oracle.run(rp, ci, x0, 1.0, 2, 99, k, **kw)
    (_, ranges, x0r, s0), (_, _, x1r, s1) = res
    assert ranges[0][0] == 0 and ranges[0][1] == ranges[1][0] and ranges[1][1] == 1000
    assert 0 < ranges[0][1] < 1000
    for x, s in ((x0r, s0), (x1r, s1)):
        np.testing.assert_allclose(x, xr, rtol=1e-9, atol=1e-9 * float(np.abs(xr).max()))
        assert s == pytest.approx(sr, rel=1e-9)


def test_vertex_ranges_cover_and_balance():
    sys.path.insert(0, ROOT)
    import numpy as np
    from paper_2011_03479_gb300 import inputs, shard
    rp, _ = inputs.rmat(12, 16, seed=5)
    n = len(rp) - 1
    work = np.diff(rp) + 1
    for world in (1, 2, 3, 4, 7):
        for block in (False, True):
            rs = shard.vertex_ranges(rp, world, block)
            assert rs[0][0] == 0 and rs[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
            if block:
                assert all(lo % 128 == 0 for lo, _ in rs)
            loads = [int(work[lo:hi].sum()) for lo, hi in rs]
            unit = 128 if block else 1
            biggest = max(int(work[i:i + unit].sum()) for i in range(0, n, unit))
            assert max(loads) - min(loads) <= 2 * biggest


def test_sharded_graph_peer_failure_gloo_world_2():
    """Failure detection on the host (no GPU involved): rank 1's engine raises
    at its second epoch, between two epochs' collectives, and the rank
    leaves.  Rank 0 must not wait for it forever: the all-reduce of its
    second epoch ends with an error (gloo reports the closed connection, a
    10 s process-group timeout bounds it otherwise), after its first epoch
    completed."""
    import _rank_worker
    sys.path.insert(0, ROOT)
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_worker.shard_peer_fails, args=(r, 2, port, q, 10)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        res = dict((r, (out, secs)) for r, out, secs in (q.get(timeout=240) for _ in procs))
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    (out1, _), (out0, secs0) = res[1], res[0]
    assert out1[0] == "injected" and out1[1] == 1
    assert out0[0] == "collective error" and out0[1] == 1, out0
    assert secs0 < 120
