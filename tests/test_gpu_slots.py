"""GPU parity of Sec. III.C's sampling policy (one non-edge sample per CSR
slot, anchored at the slot's row) against the FP64 oracle: samples bit-exact,
the FP32 epoch within the per-step bar of the per-vertex form, every launch
shape, the batched form, and the final loss of a full run within 1%.
"""
import numpy as np
import pytest

from conftest import gpu_available

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

TOL = 1e-4


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
def rmat_s12():
    from paper_2011_03479_gb300 import inputs
    return inputs.rmat(12, 16, seed=77)


def _rows_err(got, ref, floor=None):
    got = np.asarray(got, np.float64).reshape(len(ref), -1)
    ref = np.asarray(ref, np.float64).reshape(len(ref), -1)
    nr = np.linalg.norm(ref, axis=1)
    scale = np.maximum(nr, 1e-6 * max(nr.mean(), 1e-300))
    if floor is not None:
        scale = np.maximum(scale, floor)
    return np.linalg.norm(got - ref, axis=1) / scale


def _epoch(B, O, rp, ci, d, x, sigma, epoch, shape=None, **kw):
    p = B.gempe_default_params(sampling=1, **kw)
    with B.gempe_create(rp, ci, d, p) as ctx:
        if shape:
            B.gempe_set_shape(ctx, **shape)
        B.gempe_set_positions(ctx, x)
        B.gempe_set_state(ctx, sigma, epoch)
        samples = B.gempe_sweep(ctx, record_samples=True)
        delta, z = B.gempe_accumulators(ctx)
        he, hn = B.gempe_histograms(ctx, p.hist_bins)
        B.gempe_update(ctx)
        xn = B.gempe_positions(ctx)
        st = B.gempe_stats(ctx)
    ref = O.epoch(rp, ci, x.astype(np.float64), sigma, epoch, p.seed, p.neg_per_vertex, per_slot=1,
                  hist_bins=p.hist_bins, hist_max=p.hist_max)
    return dict(samples=samples, delta=delta, z=z, he=he, hn=hn, xn=xn, st=st, ref=ref)


def _check(r):
    ref = r["ref"]
    np.testing.assert_array_equal(r["samples"], ref["samples"])
    assert _rows_err(r["delta"], ref["delta"], 1e-2 * ref["abs_terms"]).max() <= TOL
    assert _rows_err(r["z"], ref["z"]).max() <= TOL
    zr = np.maximum(ref["z"], 1e-300)
    step = np.maximum(np.linalg.norm(ref["delta"].reshape(len(zr), -1), axis=1) / zr, 1e-2 * ref["abs_terms"] / zr)
    assert _rows_err(r["xn"], ref["x_new"], step).max() <= TOL
    assert r["he"].sum() == pytest.approx(ref["hist_e"].sum())
    assert r["hn"].sum() == pytest.approx(ref["hist_n"].sum(), rel=1e-5)


@pytest.mark.parametrize("d", [1, 2, 3, 4, 8, 16, 64])
def test_per_slot_epoch_parity(B, O, rmat_s12, d):
    rp, ci = rmat_s12
    n = len(rp) - 1
    x = (np.random.default_rng(50 + d).standard_normal((n, d)) * 1.1).astype(np.float32)
    r = _epoch(B, O, rp, ci, d, x, 0.8, 4)
    _check(r)
    assert r["st"]["used"] == r["ref"]["accepted"]


@pytest.mark.parametrize("d,shape", [(2, dict(unit_pairs=64)), (2, dict(kernel=1, edge_chunk=16)),
                                     (2, dict(kernel=1, edge_chunk=64)), (16, dict(lanes=4, edge_chunk=32)),
                                     (64, dict(lanes=16, edge_chunk=128))])
def test_per_slot_every_shape(B, O, rmat_s12, d, shape):
    rp, ci = rmat_s12
    n = len(rp) - 1
    x = (np.random.default_rng(70 + d).standard_normal((n, d))).astype(np.float32)
    _check(_epoch(B, O, rp, ci, d, x, 0.9, 2, shape=shape))


def test_per_slot_batch_equals_alone(B):
    from paper_2011_03479_gb300 import inputs
    gs = inputs.sbm_batch(6, 60, 1200, dims=(2, 16), seed=7300)
    p = B.gempe_default_params(sampling=1)
    with B.gempe_batch_create([(g["row_ptr"], g["col_idx"], g["d"]) for g in gs], p) as b:
        B.gempe_batch_step(b, 3)
        got = [B.gempe_batch_stats(b, q) for q in range(len(gs))]
    for q, g in enumerate(gs):
        pa = B.gempe_default_params(sampling=1, seed=p.seed ^ q)
        with B.gempe_create(g["row_ptr"], g["col_idx"], g["d"], pa) as ctx:
            B.gempe_step(ctx, 3)
            st = B.gempe_stats(ctx)
        for f in ("accepted", "rejected", "exhausted", "draws", "used", "epoch"):
            assert got[q][f] == st[f], f"graph {q}: {f}"


def test_per_slot_full_run_loss(B, O, sbm_1000):
    """200 epochs of the SBM drawing with the paper's policy: final sampled PE
    (scored by the oracle's estimator) within 1% of the oracle's run."""
    rp, ci = sbm_1000["row_ptr"], sbm_1000["col_idx"]
    p = B.gempe_default_params(sampling=1)
    with B.gempe_create(rp, ci, 2, p) as ctx:
        x0 = B.gempe_positions(ctx)
        B.gempe_step(ctx, 200)
        x = B.gempe_positions(ctx)
        s, _ = B.gempe_get_state(ctx)
    xr, sr, _ = O.run(rp, ci, x0, 1.0, 200, p.seed, 5, per_slot=1)
    pe_gpu = O.loss_sampled(rp, ci, x.astype(np.float64), s, 200, p.seed, 16)
    pe_ref = O.loss_sampled(rp, ci, xr, sr, 200, p.seed, 16)
    assert pe_gpu == pytest.approx(pe_ref, rel=0.01)
