"""GPU tests of the serving form: jobs admitted by device-memory budget and
run with continuous batching (several jobs' epochs in flight at once).

Each job must give the same result in the mix as alone (gempe_create +
gempe_step with the job's seed): the sampled pair count exactly, positions
and the final slope up to FP32 summation order.  Admission must respect the
budget, and failures (a job over budget, an invalid graph) must be reported
without stopping the other jobs.
"""
import numpy as np
import pytest

from conftest import gpu_available

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module")
def B():
    from paper_2011_03479_gb300 import binding
    binding.load()
    return binding


@pytest.fixture(scope="module")
def jobs():
    from paper_2011_03479_gb300 import inputs
    rng = np.random.default_rng(5000)
    out = []
    for q in range(10):
        scale = int(rng.integers(7, 12))
        ef = int(rng.integers(8, 17))
        rp, ci = inputs.rmat(scale, ef, seed=5001 + q)
        out.append(dict(row_ptr=rp, col_idx=ci, d=int(rng.choice([2, 32, 128])),
                        epochs=int(rng.integers(12, 40)), seed=0x5E5E0000 + q))
    return out


def _alone(B, j, **kw):
    p = B.gempe_default_params(seed=j["seed"], neg_per_vertex=10, **kw)
    with B.gempe_create(j["row_ptr"], j["col_idx"], j["d"], p) as ctx:
        B.gempe_step(ctx, j["epochs"])
        x = B.gempe_positions(ctx)
        st = B.gempe_stats(ctx)
    return x, st


def test_serve_mix_equals_alone(B, jobs):
    p = B.gempe_default_params(neg_per_vertex=10)
    with B.gempe_server_create(8 << 30, max_jobs=4, params=p) as srv:
        ids = [B.gempe_server_submit(srv, j["row_ptr"], j["col_idx"], j["d"], j["epochs"], j["seed"]) for j in jobs]
        infos = [B.gempe_server_wait(srv, i, 120000) for i in ids]
        xs = [B.gempe_server_result(srv, i) for i in ids]
        stats = B.gempe_server_stats(srv)
    assert stats["completed"] == len(jobs) and stats["failed"] == 0
    # the jobs overlapped on the device: some job started before another finished
    iv = sorted((inf["admit_ns"], inf["done_ns"]) for inf in infos)
    assert any(iv[q + 1][0] < iv[q][1] for q in range(len(iv) - 1))
    for j, inf, x in zip(jobs, infos, xs):
        assert inf["state"] == 2 and inf["epochs_done"] == j["epochs"]
        xa, sa = _alone(B, j)
        m = len(j["col_idx"]) // 2
        assert inf["pairs"] == j["epochs"] * m + sa["used"], "the same samples alone and in the mix"
        scale = max(np.abs(xa).max(), 1e-30)
        err = np.abs(x.astype(np.float64) - xa).max() / scale
        assert err <= 1e-3, f"job d={j['d']} epochs={j['epochs']}: {err:.2e}"
        assert inf["sigma"] == pytest.approx(sa["sigma"], rel=1e-3)


def test_serve_budget_bounds_running_jobs(B, jobs):
    """A budget that fits the largest job plus half the smallest: at every
    admission the jobs running together fit in the budget, admission keeps
    arrival order, and the peak reservation stays in the budget."""
    p = B.gempe_default_params(neg_per_vertex=10)
    sel = jobs[:6]
    sizes = [B.gempe_job_bytes(len(j["row_ptr"]) - 1, len(j["col_idx"]), j["d"], p) for j in sel]
    budget = max(sizes) + min(sizes) // 2
    with B.gempe_server_create(budget, max_jobs=8, params=p) as srv:
        ids = [B.gempe_server_submit(srv, j["row_ptr"], j["col_idx"], j["d"], j["epochs"], j["seed"]) for j in sel]
        infos = [B.gempe_server_wait(srv, i, 120000) for i in ids]
        for i in ids:
            B.gempe_server_result(srv, i)
        stats = B.gempe_server_stats(srv)
    for a, b in zip(infos, infos[1:]):
        assert b["admit_ns"] >= a["admit_ns"]           # arrival order
    for q, inf in enumerate(infos):
        t = inf["admit_ns"]
        running = sum(sz for sz, o in zip(sizes, infos) if o["admit_ns"] <= t < o["done_ns"])
        assert running <= budget
        assert inf["device_bytes"] == sizes[q]
    assert stats["peak_bytes_in_use"] <= budget and stats["bytes_in_use"] == 0


def test_serve_failures_reported(B, jobs):
    p = B.gempe_default_params(neg_per_vertex=10)
    j = jobs[0]
    need = B.gempe_job_bytes(len(j["row_ptr"]) - 1, len(j["col_idx"]), j["d"], p)
    with B.gempe_server_create(need - 1, max_jobs=2, params=p) as srv:
        with pytest.raises(B.GempeError) as ei:
            B.gempe_server_submit(srv, j["row_ptr"], j["col_idx"], j["d"], 5, 1)
        assert ei.value.status == -7
    with B.gempe_server_create(1 << 30, max_jobs=2, params=p) as srv:
        bad = B.gempe_server_submit(srv, np.array([0, 1, 1], np.int32), np.array([1], np.int32), 2, 5, 1)
        good = B.gempe_server_submit(srv, j["row_ptr"], j["col_idx"], j["d"], 5, 2)
        with pytest.raises(B.GempeError) as ei:
            B.gempe_server_wait(srv, bad, 60000)
        assert ei.value.status == -2
        assert B.gempe_server_wait(srv, good, 60000)["state"] == 2
        B.gempe_server_result(srv, good)
        with pytest.raises(B.GempeError):
            B.gempe_server_result(srv, bad)
        st = B.gempe_server_stats(srv)
        assert st["completed"] == 1 and st["failed"] == 1
