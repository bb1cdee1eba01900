"""GPU parity at the benchmark workloads' full sizes, in the launch
configuration bench.py times, on outputs the oracle computes one by one.

ba-n1m-m8 (n = 10^6, m ~ 8 * 10^6, d = 64, block sampling 128 x 64), in
both forms the benchmark times: BF16 positions on the tensor-core tiles and
the plain FP32 run on the FP32 tiles.  One epoch from seeded positions.  For
a sample of vertices (the highest-degree hubs, the ragged last tile, the
first vertices and random ones) the block masks are bit-exact and y - z x,
z and the step are within the per-step bar of the form (BF16: 1e-2, floored
at 3e-2 of the size of the vertex's pair terms where they cancel; FP32:
1e-4, floored at 1e-2 of it), against the oracle's Eq. 3 for those vertices
alone.

sbm-batch-256 (256 SBM graphs, d in {2, 16, 64}, autotuned launch shapes,
FP32): one epoch of the whole batch as one CUDA-graph launch.  For sampled
graphs (the smallest and the largest of each dimension) the positions after
the epoch are within the FP32 bar (1e-4 of the larger of the position and
the step) against the oracle's whole epoch of that graph, and the sampled
non-edges consumed match its count exactly.

The R-MAT workload (rmat-s16-ef16) is checked whole, every vertex, in
test_gpu_parity.py.
"""
import numpy as np
import pytest

from conftest import gpu_available

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

TOL32 = 1e-4
TOL16 = 1e-2


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


def _err_rows(got, ref, floor=None):
    """Per-row ||got - ref|| / max(||ref||, 1e-6 mean ||ref||[, floor])."""
    got = np.asarray(got, np.float64).reshape(len(ref), -1)
    ref = np.asarray(ref, np.float64).reshape(len(ref), -1)
    nr = np.linalg.norm(ref, axis=1)
    scale = np.maximum(nr, 1e-6 * max(nr.mean(), 1e-300))
    if floor is not None:
        scale = np.maximum(scale, np.asarray(floor, np.float64))
    return np.linalg.norm(got - ref, axis=1) / scale


@pytest.mark.parametrize("precision,kernel", [(1, 0), (0, 0), (1, 2), (0, 2)],
                         ids=["bf16-tcgen05-tiles", "fp32-tiles", "bf16-beside", "fp32-beside"])
def test_ba_1m_tiles_sampled_vertices(B, O, precision, kernel):
    from paper_2011_03479_gb300 import inputs
    w = inputs.ba_1m()
    rp, ci, d = w["row_ptr"], w["col_idx"], 64
    n = len(rp) - 1
    sigma, epoch = 0.7, 9
    x = (np.random.default_rng(5).normal(size=(n, d)) * 0.7).astype(np.float32)
    p = B.gempe_default_params(neg_per_vertex=w["k"], seed=inputs.EMBED_SEED, block_partners=64,
                               precision=precision)
    with B.gempe_create(rp, ci, d, p) as ctx:
        B.gempe_set_shape(ctx, kernel=kernel)
        B.gempe_set_positions(ctx, x)
        B.gempe_set_state(ctx, sigma, epoch)
        masks = B.gempe_sweep(ctx, record_samples=True)
        delta, z = B.gempe_accumulators(ctx)
        B.gempe_update(ctx)
        xn = B.gempe_positions(ctx)

    deg = np.diff(rp)
    n_tiles = (n + 127) // 128
    rng = np.random.default_rng(11)
    query = np.unique(np.concatenate([np.argsort(deg)[-8:], [0, 1, 2, n - 1, n - 2, 128 * (n_tiles - 1)],
                                      rng.choice(n, 200, replace=False)])).astype(np.int32)
    # block masks: partner p of the vertex's tile, -1 where it is the vertex or a neighbour
    for v in query:
        parts = O.block_partners(n, int(v) // 128, epoch, p.seed, 64)
        exp = [(-1 if (g == v or O.is_edge(rp, ci, v, g)) else g) for g in parts.tolist()]
        np.testing.assert_array_equal(masks[v], exp, err_msg=f"vertex {v}")

    ref = O.vertex_terms(rp, ci, x.astype(np.float64), sigma, epoch, p.seed, 0, query,
                         block_partners=64, tile_vertices=128)
    zr = np.maximum(ref["z"], 1e-300)
    # BF16: 1e-2 floored at 3e-2 of the term sizes; FP32: 1e-4 floored at 1e-2 of them
    tol, floor = (TOL16, 3e-2) if precision else (TOL32, 1e-2)
    e_delta = _err_rows(delta[query], ref["delta"], floor * ref["abs_terms"])
    e_z = _err_rows(z[query], ref["z"])
    x0 = x[query].astype(np.float64)
    e_step = _err_rows(xn[query].astype(np.float64) - x0, ref["x_new"] - x0, floor * ref["abs_terms"] / zr)
    print(f"BA 1M precision {precision} tiles, {len(query)} vertices: delta {e_delta.max():.2e} "
          f"z {e_z.max():.2e} step {e_step.max():.2e}")
    assert e_delta.max() <= tol and e_z.max() <= tol and e_step.max() <= tol


def test_batch_256_sampled_graphs(B, O):
    from paper_2011_03479_gb300 import inputs
    w = inputs.sbm_batch_256()
    graphs, k = w["graphs"], w["k"]
    p = B.gempe_default_params(neg_per_vertex=k, seed=inputs.EMBED_SEED, autotune=1)
    picks = []
    for d in (2, 16, 64):
        idx = [q for q, g in enumerate(graphs) if g["d"] == d]
        sizes = [len(graphs[q]["row_ptr"]) - 1 for q in idx]
        picks += [idx[int(np.argmin(sizes))], idx[int(np.argmax(sizes))]]
    with B.gempe_batch_create([(g["row_ptr"], g["col_idx"], g["d"]) for g in graphs], p) as b:
        B.gempe_batch_step(b, 1)
        for q in picks:
            g = graphs[q]
            rp, ci, d = g["row_ptr"], g["col_idx"], g["d"]
            n = len(rp) - 1
            key = p.seed ^ q
            x0 = O.init_positions(n, d, key).astype(np.float64)
            ref = O.epoch(rp, ci, x0, 1.0, 0, key, k)
            xn = B.gempe_batch_positions(b, q).astype(np.float64)
            st = B.gempe_batch_stats(b, q)
            # x_new judged against max(|x_new|, |delta| / z, 1e-2 A / z): the
            # position, the step, and the size of the step's terms where they
            # cancel (as in the per-step tests)
            zr = np.maximum(ref["z"], 1e-300)
            floor = np.maximum(np.linalg.norm(ref["delta"], axis=1) / zr, 1e-2 * ref["abs_terms"] / zr)
            err = _err_rows(xn, ref["x_new"], floor)
            print(f"graph {q} (n = {n}, d = {d}): step {err.max():.2e}")
            assert err.max() <= TOL32, f"graph {q} (n = {n}, d = {d})"
            assert st["epoch"] == 1
            assert st["used"] == ref["accepted"], f"graph {q}"
