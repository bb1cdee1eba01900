"""GPU parity on the method's degenerate inputs and at the largest dimension,
in every sampling form.

Degenerate inputs:

- a graph without edges (only sampled non-edges move the vertices; in the
  per-slot policy nothing moves at all and both histograms stay empty);
- the smallest graph, two vertices and one edge (in block sampling every
  partner of the one tile is the anchor itself or its neighbour: all 64
  pairs of each row masked);
- a star whose centre is the only vertex of the last tile (n = 129): the
  centre is adjacent to every other vertex, so each of its draws is
  rejected until the sample is dropped, and every partner of its one-vertex
  tile is masked.

The largest dimension, d = 256 (one lane group of 32 lanes per vertex), in
the per-vertex, per-slot and block forms with FP32 and BF16 positions (the
block samples go through the pair sweep there, as at d = 8 and, with BF16
positions, at d = 128: those two are checked as well).

Each epoch is compared with the oracle's: sampled pairs bit-exact, per-step
FP32 results under the FP32 bar (1e-4, the cancellation floor at 1e-2 of the
size A_i of a vertex's pair terms), the BF16 form against the oracle run on
the BF16-rounded positions under the bar its own roundings allow (2^-8 of
each tile term), and the refitted slope against the oracle's fit of the same
histograms (on separable histograms, where any slope with a negligible
entropy minimises it, by the entropy at the slope).
"""
import numpy as np
import pytest

from conftest import bf16_round, gpu_available

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

TOL = 1e-4
U16 = 2.0 ** -8   # BF16 unit roundoff


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


def _csr(rows):
    rp = np.cumsum([0] + [len(r) for r in rows]).astype(np.int32)
    ci = np.array([j for r in rows for j in r], dtype=np.int32)
    return rp, ci


GRAPHS = {
    "edgeless": _csr([[] for _ in range(300)]),
    "one-edge": _csr([[1], [0]]),
    "star-lone-tile": _csr([[128] for _ in range(128)] + [list(range(128))]),
}

FORMS = {
    "vertex-d2": (2, dict(neg_per_vertex=5)),
    "vertex-d16": (16, dict(neg_per_vertex=5)),
    "slot-d2": (2, dict(sampling=1)),
    "slot-d16": (16, dict(sampling=1)),
    "block-fp32-d16": (16, dict(block_partners=64)),
    "block-fp32-d64": (64, dict(block_partners=64)),
    "block-bf16-d16": (16, dict(block_partners=64, precision=1)),
    "block-bf16-d64": (64, dict(block_partners=64, precision=1)),
}


def _expected_block_samples(rp, ci, parts):
    n = len(rp) - 1
    out = np.empty((n, parts.shape[1]), dtype=np.int32)
    for i in range(n):
        row = set(ci[rp[i]:rp[i + 1]].tolist())
        out[i] = [(-1 if (g == i or g in row) else g) for g in parts[i // 128].tolist()]
    return out


def _epoch_against_oracle(B, O, rp, ci, d, kw, label, x=None):
    """One epoch on the GPU and the oracle's from the same positions x
    (default: normal, 0.9 per coordinate; rounded to BF16 for the oracle in
    the BF16 form), checked under the bars above; returns the per-vertex step
    mask (z_i >= z_min), the histograms, the slope and the oracle's epoch."""
    n = len(rp) - 1
    p = B.gempe_default_params(**kw)
    if x is None:
        x = (np.random.default_rng(n + d).normal(size=(n, d)) * 0.9).astype(np.float32)
    bf16 = p.precision == 1
    xr = bf16_round(x) if bf16 else x
    with B.gempe_create(rp, ci, d, p) as ctx:
        B.gempe_set_positions(ctx, x)
        B.gempe_set_state(ctx, 0.8, 3)
        samples = B.gempe_sweep(ctx, record_samples=True)
        delta, z = B.gempe_accumulators(ctx)
        he, hn = B.gempe_histograms(ctx, p.hist_bins)
        B.gempe_update(ctx)
        xn = B.gempe_positions(ctx)
        sigma, _ = B.gempe_get_state(ctx)
        stats = B.gempe_stats(ctx)
    ref = O.epoch(rp, ci, xr.astype(np.float64), 0.8, 3, p.seed, p.neg_per_vertex, mu=p.mu,
                  max_retries=p.max_retries, symmetric=p.symmetric_neg, w_formula=p.w_formula,
                  clamp_neg_d=p.clamp_neg_d, z_min=p.z_min, hist_bins=p.hist_bins, hist_max=p.hist_max,
                  block_partners=p.block_partners, tile_vertices=128, per_slot=p.sampling)
    # the sampled pairs
    if p.block_partners:
        np.testing.assert_array_equal(samples, _expected_block_samples(rp, ci, ref["partners"]))
    else:
        np.testing.assert_array_equal(samples, ref["samples"])
    assert stats["used"] == ref["accepted"]
    # per-step sums, weights and positions
    a_i, zr = ref["abs_terms"], ref["z"]
    # the BF16 rounding of the coefficients happens only in the tensor-core
    # tiles (d = 16, 32, 64); the pair sweep keeps them in FP32
    u = U16 if bf16 and p.block_partners and d in (16, 32, 64) else 0.0
    err_d = np.linalg.norm(np.asarray(delta, np.float64) - ref["delta"], axis=1)
    bar_d = u * a_i + TOL * np.maximum(np.linalg.norm(ref["delta"], axis=1), 1e-2 * a_i)
    assert (err_d <= bar_d).all(), np.max(err_d - bar_d)
    err_z = np.abs(np.asarray(z, np.float64) - zr)
    assert (err_z <= (u + TOL) * zr).all(), np.max(err_z / np.maximum(zr, 1e-300))
    moved = zr >= p.z_min
    assert np.array_equal(xn[~moved], x[~moved])   # z below z_min: the vertex stays
    step = xn[moved].astype(np.float64) - x[moved].astype(np.float64)
    step_ref = ref["x_new"][moved] - xr[moved].astype(np.float64)
    zg = np.asarray(z, np.float64)[moved]
    bar_x = (bar_d[moved] + np.linalg.norm(step_ref, axis=1) * (u + TOL) * zr[moved]) / zg \
        + 2.0 ** -22 * np.linalg.norm(xn[moved].astype(np.float64), axis=1)
    assert (np.linalg.norm(step - step_ref, axis=1) <= bar_x).all()
    # histograms and the slope refitted from them
    assert he.sum() == len(ci) // 2
    assert hn.sum() == pytest.approx(ref["hist_n"].sum(), rel=1e-5, abs=1e-3)
    he64, hn64 = he.astype(np.float64), hn.astype(np.float64)
    s_ref = O.sigma_fit(he64, hn64)
    pe = lambda s: O.hist_pe(he64, hn64, p.hist_max, p.mu, s)   # noqa: E731
    if pe(s_ref) <= 1e-12 * pe(1e3):
        # separable histograms (every edge below mu, every non-edge above it):
        # the entropy falls towards 0 as sigma -> 0 and every sigma at which it
        # has become negligible is a minimiser; the FP64 bisection stops where
        # its terms underflow, the FP32 search where its own do
        assert pe(sigma) <= 1e-12 * pe(1e3)
    else:
        assert sigma == pytest.approx(s_ref, rel=TOL)
    print(f"{label}: delta {np.max(err_d / np.maximum(bar_d, 1e-300)):.2f} of its bar, "
          f"sigma {sigma:.4g}, moved {int(moved.sum())} of {n}")
    return dict(moved=moved, he=he, hn=hn, sigma=sigma, ref=ref, s_ref=s_ref)


@pytest.mark.parametrize("form", list(FORMS))
@pytest.mark.parametrize("graph", list(GRAPHS))
def test_degenerate_graph_epoch(B, O, graph, form):
    rp, ci = GRAPHS[graph]
    d, kw = FORMS[form]
    r = _epoch_against_oracle(B, O, rp, ci, d, kw, f"{graph} {form}")
    if graph == "edgeless" and kw.get("sampling") == 1:
        # no edges and no samples: nothing moves, both histograms stay empty
        assert not r["moved"].any() and r["he"].sum() == 0 and r["hn"].sum() == 0
        assert r["sigma"] == pytest.approx(1e3)


WIDE = {
    "vertex-fp32-d256": (256, dict(neg_per_vertex=5)),
    "vertex-bf16-d256": (256, dict(neg_per_vertex=5, precision=1)),
    "slot-fp32-d256": (256, dict(sampling=1)),
    "block-fp32-d256": (256, dict(block_partners=64)),
    "block-bf16-d256": (256, dict(block_partners=64, precision=1)),
    "block-bf16-d128": (128, dict(block_partners=64, precision=1)),
    "block-bf16-d8": (8, dict(block_partners=64, precision=1)),
}


@pytest.mark.parametrize("form", list(WIDE))
def test_largest_dimension_and_sweep_block_forms(B, O, sbm_1000, form):
    """d = 256 in every form, and the BF16 block samples that the pair sweep
    evaluates (d = 8, 128, 256: no tensor-core tiles there, so the BF16 form
    is FP32 arithmetic on the rounded positions and meets the FP32 bar
    against the oracle on those positions)."""
    d, kw = WIDE[form]
    _epoch_against_oracle(B, O, sbm_1000["row_ptr"], sbm_1000["col_idx"], d, kw, f"sbm-1000 {form}")


CLUSTERED = {
    "vertex-fp32-d64": (64, dict(neg_per_vertex=5)),
    "vertex-bf16-d64": (64, dict(neg_per_vertex=5, precision=1)),
    "slot-fp32-d64": (64, dict(sampling=1)),
    "block-fp32-d16": (16, dict(block_partners=64)),
    "block-fp32-d64": (64, dict(block_partners=64)),
    "block-fp32-d128": (128, dict(block_partners=64)),
    "block-bf16-d16": (16, dict(block_partners=64, precision=1)),
    "block-bf16-d64": (64, dict(block_partners=64, precision=1)),
    "block-fp32-d256": (256, dict(block_partners=64)),
}


@pytest.mark.parametrize("form", list(CLUSTERED))
def test_clustered_positions(B, O, sbm_1000, form):
    """Positions of an embedding that has found the SBM's four blocks: each
    block around its own centre (centres about 3 apart, points about 0.8
    from their block mates), so edges and the many intra-block non-edges lie
    below mu = 1.5 and inter-block pairs above it.  Unlike spread random
    positions at large d, whose pairs all sit far in the tails of the pair
    terms (and in the histograms' last bin), these exercise the middle of
    the Mills-ratio table on both sides of mu in the tile kernels and the
    sweeps, and give histograms over 70 to 400 bins with a slope inside the
    bracket: the edge histogram within a few rounding moves of the oracle's
    and the slope within 1e-4."""
    d, kw = CLUSTERED[form]
    rp, ci = sbm_1000["row_ptr"], sbm_1000["col_idx"]
    n = len(rp) - 1
    rng = np.random.default_rng(500 + d)
    centre = rng.normal(size=(4, d)) * (3.0 / np.sqrt(2 * d))
    x = (centre[np.arange(n) // 250] + rng.normal(size=(n, d)) * (0.8 / np.sqrt(2 * d))).astype(np.float32)
    r = _epoch_against_oracle(B, O, rp, ci, d, kw, f"sbm-1000 clustered {form}", x=x)
    ref = r["ref"]
    assert np.count_nonzero(r["he"]) > 50 and 0.1 < r["s_ref"] < 10.0
    # a pair may land in a neighbouring bin when its FP32 distance rounds across a bin edge
    assert np.abs(r["he"] - ref["hist_e"]).sum() <= 8
    assert r["sigma"] == pytest.approx(r["s_ref"], rel=TOL)
