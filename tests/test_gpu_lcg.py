"""GPU parity of Sec. III.C's random number generator (rng = 1): the 32-bit
LCG with multiplier 1103515245 and increment 1, one state per sample slot
seeded from Philox and advanced before every draw, vertices by Fig. 2's FP32
float trick.  Sampled partners bit-exact against the FP64 oracle in both
sampling policies, with the exact edge set and with the byte map (whose
address wraps 32 bits at n > 65,536); sampler counts exact over a run; the
inspection sampler; every graph of a batch as alone; the final loss of a
full run within 1% of the oracle's.
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
def O():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="module")
def rmat_s12():
    from paper_2011_03479_gb300 import inputs
    return inputs.rmat(12, 16, seed=77)


@pytest.mark.parametrize("sampling", [0, 1], ids=["k-per-vertex", "per-slot"])
@pytest.mark.parametrize("kw", [dict(), dict(membership=1, bytemap_log2=19, rename_every=2)],
                         ids=["exact-set", "byte-map"])
def test_lcg_samples_bit_exact(B, O, rmat_s12, sampling, kw):
    rp, ci = rmat_s12
    n = len(rp) - 1
    p = B.gempe_default_params(sampling=sampling, neg_per_vertex=10, rng=1, **kw)
    x = np.random.default_rng(4).standard_normal((n, 2)).astype(np.float32)
    with B.gempe_create(rp, ci, 2, p) as ctx:
        B.gempe_set_positions(ctx, x)
        B.gempe_set_state(ctx, 0.9, 5)
        s5 = B.gempe_sweep(ctx, record_samples=True)
        delta, z = B.gempe_accumulators(ctx)
        B.gempe_update(ctx)
        st = B.gempe_stats(ctx)
        s6 = B.gempe_sweep(ctx, record_samples=True)
        B.gempe_update(ctx)
    refs = [O.epoch(rp, ci, x.astype(np.float64), 0.9, e, p.seed, 10, per_slot=sampling, rng=1, **kw)
            for e in (5, 6)]
    np.testing.assert_array_equal(s5, refs[0]["samples"])
    np.testing.assert_array_equal(s6, refs[1]["samples"])
    for f in ("accepted", "rejected", "exhausted", "false_pos"):
        assert st[f] == refs[0][f] + refs[1][f], f
    # the epoch's sums with these samples (FP32 bar, floored where terms cancel)
    ref = refs[0]
    nr = np.linalg.norm(ref["delta"], axis=1)
    scale = np.maximum.reduce([nr, 1e-6 * np.full_like(nr, nr.mean()), 1e-2 * ref["abs_terms"]])
    err = np.linalg.norm(delta.astype(np.float64) - ref["delta"], axis=1) / scale
    assert err.max() <= 1e-4
    np.testing.assert_allclose(z, ref["z"], rtol=1e-4)


def test_lcg_differs_from_philox_and_wraps_32_bits(B, O):
    """n = 131,072: the byte map's address wraps 32 bits; the LCG's samples
    differ from the Philox draws of the same seed and match the oracle."""
    from paper_2011_03479_gb300 import inputs
    rp, ci = inputs.rmat(17, 8, seed=178)
    n = len(rp) - 1
    out = {}
    for rng in (0, 1):
        p = B.gempe_default_params(neg_per_vertex=6, membership=1, bytemap_log2=22, rng=rng)
        with B.gempe_create(rp, ci, 2, p) as ctx:
            B.gempe_set_state(ctx, 1.0, 3)
            out[rng] = B.gempe_sweep(ctx, record_samples=True)
            B.gempe_update(ctx)
    ref = O.epoch(rp, ci, np.zeros((n, 2)), 1.0, 3, p.seed, 6, membership=1, bytemap_log2=22, rng=1)
    np.testing.assert_array_equal(out[1], ref["samples"])
    assert (out[0] != out[1]).mean() > 0.9


def test_lcg_run_counts_and_inspection(B, O, rmat_s12):
    rp, ci = rmat_s12
    n = len(rp) - 1
    p = B.gempe_default_params(neg_per_vertex=8, rng=1)
    with B.gempe_create(rp, ci, 4, p) as ctx:
        B.gempe_step(ctx, 9)
        st = B.gempe_stats(ctx)
        insp = B.gempe_sample(ctx)            # the epoch's samples of epoch 9, exact set
    tot = dict(accepted=0, rejected=0, exhausted=0)
    for e in range(10):                       # the run samples one epoch ahead
        r = O.epoch(rp, ci, np.zeros((n, 1)), 1.0, e, p.seed, 8, rng=1)
        for f in tot:
            tot[f] += r[f]
        if e == 9:
            np.testing.assert_array_equal(insp, r["samples"])
    for f in tot:
        assert st[f] == tot[f], f


def test_lcg_batch_equals_alone(B):
    from paper_2011_03479_gb300 import inputs
    gs = inputs.sbm_batch(5, 60, 1500, dims=(2, 16), seed=7410)
    for sampling in (0, 1):
        p = B.gempe_default_params(rng=1, sampling=sampling)
        with B.gempe_batch_create([(g["row_ptr"], g["col_idx"], g["d"]) for g in gs], p) as b:
            B.gempe_batch_step(b, 4)
            got = [B.gempe_batch_stats(b, q) for q in range(len(gs))]
        for q, g in enumerate(gs):
            pa = B.gempe_default_params(seed=p.seed ^ q, rng=1, sampling=sampling)
            with B.gempe_create(g["row_ptr"], g["col_idx"], g["d"], pa) as ctx:
                B.gempe_step(ctx, 4)
                st = B.gempe_stats(ctx)
            for f in ("accepted", "rejected", "exhausted", "used", "epoch"):
                assert got[q][f] == st[f], f"graph {q}: {f}"


def test_lcg_full_run_loss(B, O, sbm_1000):
    """200 epochs of the SBM drawing with the LCG: the final sampled PE within
    1% of the oracle's run with the same generator."""
    rp, ci = sbm_1000["row_ptr"], sbm_1000["col_idx"]
    p = B.gempe_default_params(rng=1)
    epochs = 200
    with B.gempe_create(rp, ci, 2, p) as ctx:
        x0 = B.gempe_positions(ctx)
        B.gempe_step(ctx, epochs)
        x = B.gempe_positions(ctx)
        sigma, _ = B.gempe_get_state(ctx)
    xr, sr, _ = O.run(rp, ci, x0.astype(np.float64), 1.0, epochs, p.seed, p.neg_per_vertex, rng=1)
    pe_gpu = O.loss_sampled(rp, ci, np.asarray(x, np.float64), sigma, epochs, p.seed, 32)
    pe_ref = O.loss_sampled(rp, ci, xr, sr, epochs, p.seed, 32)
    assert pe_gpu == pytest.approx(pe_ref, rel=0.01)
