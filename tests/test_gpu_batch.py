"""GPU tests of the batched form: many graphs of mixed dimension stepped
together by one CUDA-graph launch per epoch.

Graph g of a batch uses the Philox key seed ^ g.  Its first epoch must match
the FP64 oracle run with that key (FP32 tolerance 1e-4, as for a single
graph); after several epochs it must match the same graph run alone: the
sampler's integer statistics exactly (same samples), positions and sigma up
to FP32 summation order.
"""
import numpy as np
import pytest

from conftest import gpu_available

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

TOL32 = 1e-4
SEED = 0x6E6D7065
INT_STATS = ("accepted", "rejected", "exhausted", "draws", "used", "epoch")


@pytest.fixture(scope="module")
def B():
    from paper_2011_03479_gb300 import binding
    binding.load()
    return binding


@pytest.fixture(scope="module")
def O():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="module")
def graphs():
    from paper_2011_03479_gb300 import inputs
    gs = inputs.sbm_batch(9, 40, 1500, dims=(2, 16, 64), seed=7000)
    # edge cases: two vertices and no edge; a path with an isolated vertex
    gs.append(dict(row_ptr=np.array([0, 0, 0], np.int32), col_idx=np.zeros(0, np.int32), d=16))
    gs.append(dict(row_ptr=np.array([0, 1, 3, 4, 4], np.int32), col_idx=np.array([1, 0, 2, 1], np.int32), d=2))
    return gs


def _err_rows(got, ref):
    got = np.asarray(got, np.float64).reshape(len(ref), -1)
    ref = np.asarray(ref, np.float64).reshape(len(ref), -1)
    nr = np.linalg.norm(ref, axis=1)
    scale = np.maximum(nr, 1e-6 * max(nr.mean(), 1e-300))
    return np.linalg.norm(got - ref, axis=1) / scale


def _batch(B, gs, **kw):
    p = B.gempe_default_params(**kw)
    return B.gempe_batch_create([(g["row_ptr"], g["col_idx"], g["d"]) for g in gs], p), p


def test_batch_first_epoch_matches_oracle(B, O, graphs):
    b, p = _batch(B, graphs, neg_per_vertex=5)
    with b:
        B.gempe_batch_step(b, 1)
        for q, g in enumerate(graphs):
            rp, ci, d = g["row_ptr"], g["col_idx"], g["d"]
            n = len(rp) - 1
            x0 = O.init_positions(n, d, SEED ^ q)
            ref = O.epoch(rp, ci, x0.astype(np.float64), 1.0, 0, SEED ^ q, 5)
            xn = B.gempe_batch_positions(b, q)
            err = _err_rows(xn, ref["x_new"]).max()
            st = B.gempe_batch_stats(b, q)
            assert err <= TOL32, f"graph {q} (n={n}, d={d}): {err:.2e}"
            assert st["epoch"] == 1
            assert st["used"] == ref["accepted"], f"graph {q}"


@pytest.mark.parametrize("precision,block", [(0, 0), (1, 0), (1, 64)])
def test_batch_equals_alone(B, graphs, precision, block):
    epochs = 4
    b, p = _batch(B, graphs, precision=precision, block_partners=block)
    with b:
        B.gempe_batch_step(b, epochs)
        got = [(B.gempe_batch_positions(b, q), B.gempe_batch_stats(b, q)) for q in range(len(graphs))]
    tol = 1e-3 if precision == 0 else 1e-2
    for q, g in enumerate(graphs):
        d = g["d"]
        wide = d >= 8
        pa = B.gempe_default_params(seed=SEED ^ q, precision=precision if wide else 0,
                                    block_partners=block if wide else 0)
        with B.gempe_create(g["row_ptr"], g["col_idx"], d, pa) as ctx:
            B.gempe_step(ctx, epochs)
            x_alone = B.gempe_positions(ctx)
            st_alone = B.gempe_stats(ctx)
        x_b, st_b = got[q]
        for f in INT_STATS:
            assert st_b[f] == st_alone[f], f"graph {q} d={d}: {f} {st_b[f]} != {st_alone[f]}"
        scale = max(np.abs(x_alone).max(), 1e-30)
        err = np.abs(x_b.astype(np.float64) - x_alone).max() / scale
        assert err <= tol, f"graph {q} d={d}: positions differ by {err:.2e} of their scale"
        assert st_b["sigma"] == pytest.approx(st_alone["sigma"], rel=tol)


def test_batch_loss_matches_alone(B, graphs):
    b, p = _batch(B, graphs)
    with b:
        B.gempe_batch_step(b, 3)
        losses = [B.gempe_batch_loss(b, q) for q in range(len(graphs))]
    for q, g in enumerate(graphs):
        with B.gempe_create(g["row_ptr"], g["col_idx"], g["d"], B.gempe_default_params(seed=SEED ^ q)) as ctx:
            B.gempe_step(ctx, 3)
            pe, s = B.gempe_loss(ctx)
        assert losses[q][0] == pytest.approx(pe, rel=1e-3, abs=1e-9), f"graph {q}"
        assert losses[q][1] == pytest.approx(s, rel=1e-3)


def test_batch_autotune_keeps_results(B, graphs):
    """The tuner changes launch shapes only: one epoch still matches the
    untuned batch within the FP32 tolerance, and the epoch state it timed
    on is left as it was."""
    b0, _ = _batch(B, graphs)
    b1, _ = _batch(B, graphs, autotune=1)
    with b0, b1:
        for d in (2, 16, 64):
            shape = B.gempe_batch_shape(b1, d)
            assert shape["graphs"] >= 1 and shape["grid"] > 0
        st1 = [B.gempe_batch_stats(b1, q) for q in range(len(graphs))]
        assert all(s["epoch"] == 0 and s["used"] == 0 for s in st1)
        B.gempe_batch_step(b0, 1)
        B.gempe_batch_step(b1, 1)
        for q in range(len(graphs)):
            x0 = B.gempe_batch_positions(b0, q)
            x1 = B.gempe_batch_positions(b1, q)
            assert _err_rows(x1, x0).max() <= TOL32, f"graph {q}"
            assert B.gempe_batch_stats(b0, q)["used"] == B.gempe_batch_stats(b1, q)["used"]
