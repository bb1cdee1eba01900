"""GPU parity of Sec. III.C's lossy membership test (the byte map with its
periodic random renaming) against the FP64 oracle: the sampled partners
bit-exact in both sampling policies, with the map rebuilt for a new
renaming period on the stream of the next epoch's sampler and on the
current one; the rejected-draw and false-positive counts exact over a run;
a map large enough that no two pairs share an address equal to the exact
test; every graph of a batch as alone; and the final loss of a full run
within 1% of the oracle's.
"""
import numpy as np
import pytest

from conftest import gpu_available

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

LOG2 = 19          # 512 KiB for ~1e5 directed edges: about one random non-edge in six collides
RENAME = 2


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


def _oracle_counts(O, rp, ci, epochs, seed, k, per_slot, log2, rename):
    n = len(rp) - 1
    tot = dict(accepted=0, rejected=0, exhausted=0, false_pos=0)
    x = np.zeros((n, 1))
    for e in epochs:
        r = O.epoch(rp, ci, x, 1.0, e, seed, k, per_slot=per_slot, membership=1, bytemap_log2=log2,
                    rename_every=rename)
        for f in tot:
            tot[f] += r[f]
    return tot


@pytest.mark.parametrize("sampling", [0, 1])
@pytest.mark.parametrize("d", [2, 16])
def test_bytemap_samples_bit_exact(B, O, rmat_s12, sampling, d):
    """set_state moves the context to epoch 5 (renaming period 2): the map is
    rebuilt before the sampler of epoch 5 (context stream) and again before
    that of epoch 6 (period 3, side stream, beside the sweep)."""
    rp, ci = rmat_s12
    n = len(rp) - 1
    p = B.gempe_default_params(sampling=sampling, neg_per_vertex=10, membership=1, bytemap_log2=LOG2,
                               rename_every=RENAME)
    x = (np.random.default_rng(3).standard_normal((n, d))).astype(np.float32)
    with B.gempe_create(rp, ci, d, p) as ctx:
        B.gempe_set_positions(ctx, x)
        B.gempe_set_state(ctx, 0.9, 5)
        samples = B.gempe_sweep(ctx, record_samples=True)
        B.gempe_update(ctx)
        st = B.gempe_stats(ctx)
        samples6 = B.gempe_sweep(ctx, record_samples=True)
        B.gempe_update(ctx)
    ref = O.epoch(rp, ci, x.astype(np.float64), 0.9, 5, p.seed, 10, per_slot=sampling, membership=1,
                  bytemap_log2=LOG2, rename_every=RENAME)
    ref6 = O.epoch(rp, ci, x.astype(np.float64), 0.9, 6, p.seed, 10, per_slot=sampling, membership=1,
                   bytemap_log2=LOG2, rename_every=RENAME)
    np.testing.assert_array_equal(samples, ref["samples"])
    np.testing.assert_array_equal(samples6, ref6["samples"])
    assert ref["false_pos"] > 0, "the map is small enough to collide"
    for f in ("accepted", "rejected", "exhausted", "false_pos"):
        assert st[f] == ref[f] + ref6[f], f


@pytest.mark.parametrize("sampling", [0, 1])
def test_bytemap_wraps_32_bits(B, O, sampling):
    """n = 131,072 (R-MAT scale 17): pi(i) n + pi(j) exceeds 2^32 for most
    pairs, so the address depends on the 32-bit wrap-around Sec. III.C
    prints; the samples of two epochs in different renaming periods are
    bit-exact and the rejected and false-positive counts exact."""
    from paper_2011_03479_gb300 import inputs
    rp, ci = inputs.rmat(17, 8, seed=177)
    n = len(rp) - 1
    assert n == 131072 and (n - 1) * n >= 1 << 32
    log2 = 22
    p = B.gempe_default_params(sampling=sampling, neg_per_vertex=10, membership=1, bytemap_log2=log2,
                               rename_every=RENAME)
    x = np.zeros((n, 2), dtype=np.float32)
    with B.gempe_create(rp, ci, 2, p) as ctx:
        B.gempe_set_positions(ctx, x)
        B.gempe_set_state(ctx, 1.0, 5)
        s5 = B.gempe_sweep(ctx, record_samples=True)
        B.gempe_update(ctx)
        st = B.gempe_stats(ctx)
        s6 = B.gempe_sweep(ctx, record_samples=True)
        B.gempe_update(ctx)
    refs = [O.epoch(rp, ci, x.astype(np.float64), 1.0, e, p.seed, 10, per_slot=sampling, membership=1,
                    bytemap_log2=log2, rename_every=RENAME) for e in (5, 6)]
    np.testing.assert_array_equal(s5, refs[0]["samples"])
    np.testing.assert_array_equal(s6, refs[1]["samples"])
    assert refs[0]["false_pos"] > 0
    for f in ("accepted", "rejected", "exhausted", "false_pos"):
        assert st[f] == refs[0][f] + refs[1][f], f


def test_bytemap_run_counts(B, O, rmat_s12):
    """Twelve epochs with a renaming every three: the sampler's counts over
    epochs 0..12 (the run samples one epoch ahead) equal the oracle's."""
    rp, ci = rmat_s12
    p = B.gempe_default_params(neg_per_vertex=8, membership=1, bytemap_log2=LOG2, rename_every=3)
    with B.gempe_create(rp, ci, 4, p) as ctx:
        B.gempe_step(ctx, 12)
        st = B.gempe_stats(ctx)
    ref = _oracle_counts(O, rp, ci, range(13), p.seed, 8, 0, LOG2, 3)
    for f in ref:
        assert st[f] == ref[f], f


def test_collision_free_map_is_exact(B, rmat_s12):
    """s >= n^2: i' n + j' < s never wraps, the address is a bijection of the
    pair, so the byte map decides exactly like the edge set."""
    from paper_2011_03479_gb300 import inputs
    rp, ci = inputs.rmat(9, 8, seed=91)
    n = len(rp) - 1
    assert n * n <= 1 << 18
    out = []
    for kw in (dict(), dict(membership=1, bytemap_log2=18, rename_every=1)):
        p = B.gempe_default_params(neg_per_vertex=10, **kw)
        with B.gempe_create(rp, ci, 2, p) as ctx:
            B.gempe_step(ctx, 5)
            out.append((B.gempe_positions(ctx), B.gempe_stats(ctx)))
    (xa, sa), (xb, sb) = out
    assert sb["false_pos"] == 0
    for f in ("accepted", "rejected", "exhausted", "used"):
        assert sa[f] == sb[f], f
    np.testing.assert_allclose(xb, xa, rtol=0, atol=1e-4 * max(np.abs(xa).max(), 1.0))


def test_bytemap_batch_equals_alone(B):
    from paper_2011_03479_gb300 import inputs
    gs = inputs.sbm_batch(5, 60, 1500, dims=(2, 16), seed=7400)
    kw = dict(membership=1, bytemap_log2=15, rename_every=2)
    p = B.gempe_default_params(**kw)
    with B.gempe_batch_create([(g["row_ptr"], g["col_idx"], g["d"]) for g in gs], p) as b:
        B.gempe_batch_step(b, 5)
        got = [B.gempe_batch_stats(b, q) for q in range(len(gs))]
    assert sum(g["false_pos"] for g in got) > 0
    for q, g in enumerate(gs):
        pa = B.gempe_default_params(seed=p.seed ^ q, **kw)
        with B.gempe_create(g["row_ptr"], g["col_idx"], g["d"], pa) as ctx:
            B.gempe_step(ctx, 5)
            st = B.gempe_stats(ctx)
        for f in ("accepted", "rejected", "exhausted", "false_pos", "used", "epoch"):
            assert got[q][f] == st[f], f"graph {q}: {f}"


def test_bytemap_full_run_loss(B, O, sbm_1000):
    """150 epochs of the SBM drawing with a 64 KiB map renamed every 10
    epochs: the final sampled PE (the oracle's estimator, exact membership)
    within 1% of the oracle's run with the same map."""
    rp, ci = sbm_1000["row_ptr"], sbm_1000["col_idx"]
    kw = dict(membership=1, bytemap_log2=16, rename_every=10)
    p = B.gempe_default_params(**kw)
    epochs = 150
    with B.gempe_create(rp, ci, 2, p) as ctx:
        x0 = B.gempe_positions(ctx)
        B.gempe_step(ctx, epochs)
        x = B.gempe_positions(ctx)
        sigma, _ = B.gempe_get_state(ctx)
        st = B.gempe_stats(ctx)
    xr, sr, rst = O.run(rp, ci, x0.astype(np.float64), 1.0, epochs, p.seed, p.neg_per_vertex,
                        membership=1, bytemap_log2=16, rename_every=10)
    assert rst["false_pos"] > 0 and st["false_pos"] >= rst["false_pos"]
    pe_gpu = O.loss_sampled(rp, ci, np.asarray(x, np.float64), sigma, epochs, p.seed, 32)
    pe_ref = O.loss_sampled(rp, ci, xr, sr, epochs, p.seed, 32)
    assert pe_gpu == pytest.approx(pe_ref, rel=0.01)
