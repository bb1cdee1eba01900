"""GPU parity of one graph split over vertex-range shards (gempe_create_shard
and the exchange of shard.py), with the shards of every rank in one process
on one GPU (shard.local_epochs: the all-reduces become plain sums).

First epoch from injected positions: the summed sums of y - z x and z and
the updated positions against the oracle's whole-graph epoch, FP32 bar
(1e-4, floored at 1e-2 of the vertex's term sizes where they cancel; BF16:
1e-2 floored at 3e-2), in the per-vertex, per-slot, block FP32 tile and
block BF16 tile forms.  Over several epochs: the shards' sampler counts add
up to those of one whole-graph context exactly, and the positions and sigma
agree with it up to the order of FP32 atomic additions.
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


def _rows_err(got, ref, floor):
    got = np.asarray(got, np.float64).reshape(len(ref), -1)
    ref = np.asarray(ref, np.float64).reshape(len(ref), -1)
    nr = np.linalg.norm(ref, axis=1)
    scale = np.maximum.reduce([nr, np.full_like(nr, 1e-6 * max(nr.mean(), 1e-300)), floor])
    return np.linalg.norm(got - ref, axis=1) / scale


FORMS = [("per-vertex-d2", 2, dict(neg_per_vertex=5), 1e-4, 1e-2),
         ("per-vertex-d16", 16, dict(neg_per_vertex=5), 1e-4, 1e-2),
         ("per-slot-d2", 2, dict(neg_per_vertex=5, sampling=1), 1e-4, 1e-2),
         ("block-fp32-d64", 64, dict(block_partners=64), 1e-4, 1e-2),
         ("block-bf16-d64", 64, dict(block_partners=64, precision=1), 1e-2, 3e-2)]


@pytest.mark.parametrize("name,d,kw,tol,floor", FORMS, ids=[f[0] for f in FORMS])
@pytest.mark.parametrize("world", [2, 3])
def test_sharded_epoch_matches_oracle(B, O, sbm_1000, name, d, kw, tol, floor, world):
    import torch
    from paper_2011_03479_gb300 import shard
    rp, ci = sbm_1000["row_ptr"], sbm_1000["col_idx"]
    n = len(rp) - 1
    p = B.gempe_default_params(**kw)
    ranges = shard.vertex_ranges(rp, world, block=bool(kw.get("block_partners")))
    x = (np.random.default_rng(d + world).normal(size=(n, d)) * 0.9).astype(np.float32)
    sigma, epoch = 0.85, 3
    s = torch.cuda.Stream()
    engines = [shard.GpuShard(rp, ci, d, lo, hi, p, stream=s) for lo, hi in ranges]
    try:
        with torch.cuda.stream(s):
            xt = torch.from_numpy(x).cuda()
            for e in engines:
                e.set_positions(xt)
                B.gempe_set_state(e.ctx, sigma, epoch)
            for e in engines:
                e.sweep()
            parts = [[t.clone() for t in e.partials()] for e in engines]
            total = [sum(q[i] for q in parts) for i in range(len(parts[0]))]
            for e in engines:
                e.set_partials([t.clone() for t in total])
                e.update()
            xn = sum(shard._own_rows_only(e.positions(), e.lo, e.hi) for e in engines).cpu().numpy()
            acc = total[0].view(n, -1).cpu().numpy()
        stats = [B.gempe_stats(e.ctx) for e in engines]
        sig = [B.gempe_get_state(e.ctx)[0] for e in engines]
    finally:
        for e in engines:
            e.close()
    ref = O.epoch(rp, ci, x.astype(np.float64), sigma, epoch, p.seed, p.neg_per_vertex,
                  block_partners=p.block_partners, per_slot=p.sampling)
    e_delta = _rows_err(acc[:, :d], ref["delta"], floor * ref["abs_terms"])
    e_z = _rows_err(acc[:, d], ref["z"], np.zeros(n))
    x0 = x.astype(np.float64)
    zr = np.maximum(ref["z"], 1e-300)
    e_step = _rows_err(xn - x0, ref["x_new"] - x0, floor * ref["abs_terms"] / zr)
    print(f"{name} over {world} shards: delta {e_delta.max():.2e} z {e_z.max():.2e} step {e_step.max():.2e}")
    assert e_delta.max() <= tol and e_z.max() <= tol and e_step.max() <= tol
    assert sum(s["used"] for s in stats) == ref["accepted"]
    assert len(set(sig)) == 1          # every shard fits the same sigma on the summed histograms


@pytest.mark.parametrize("d,kw", [(2, dict(neg_per_vertex=10)), (64, dict(block_partners=64))],
                         ids=["rmat-d2", "rmat-d64-block"])
def test_sharded_run_matches_whole_graph(B, sbm_1000, d, kw):
    """Six epochs over three shards against one whole-graph context."""
    import torch
    from paper_2011_03479_gb300 import inputs, shard
    rp, ci = inputs.rmat(12, 16, seed=77)
    p = B.gempe_default_params(**kw)
    ranges = shard.vertex_ranges(rp, 3, block=bool(kw.get("block_partners")))
    with B.gempe_create(rp, ci, d, p) as whole:
        x0 = B.gempe_positions(whole)
        for _ in range(6):
            B.gempe_sweep(whole)
            B.gempe_update(whole)
        xw = B.gempe_positions(whole)
        sw = B.gempe_stats(whole)
    s = torch.cuda.Stream()
    engines = [shard.GpuShard(rp, ci, d, lo, hi, p, stream=s) for lo, hi in ranges]
    try:
        shard.local_epochs(engines, 6)
        with torch.cuda.stream(s):
            xs = engines[0].positions().cpu().numpy()
            for e in engines[1:]:
                np.testing.assert_array_equal(e.positions().cpu().numpy(), xs)
        st = [B.gempe_stats(e.ctx) for e in engines]
        ss = B.gempe_get_state(engines[0].ctx)[0]
    finally:
        for e in engines:
            e.close()
    assert x0.shape == xs.shape
    for f in ("accepted", "rejected", "exhausted", "used"):
        assert sum(s[f] for s in st) == sw[f], f
    assert ss == pytest.approx(sw["sigma"], rel=1e-3)
    scale = max(float(np.abs(xw).max()), 1e-30)
    assert float(np.abs(xs.astype(np.float64) - xw).max()) / scale <= 1e-3


def test_shard_arguments_checked(B, sbm_1000):
    rp, ci = sbm_1000["row_ptr"], sbm_1000["col_idx"]
    for lo, hi, kw in ((0, 0, {}), (5, 3, {}), (0, 1001, {}), (-1, 10, {}),
                       (100, 1000, dict(block_partners=64)), (0, 300, dict(block_partners=64))):
        with pytest.raises(B.GempeError) as err:
            B.gempe_create_shard(rp, ci, 16, lo, hi, B.gempe_default_params(**kw))
        assert err.value.status == -1
    with B.gempe_create(rp, ci, 2, B.gempe_default_params()) as ctx:
        import torch
        with pytest.raises(B.GempeError, match="not a shard"):
            B.gempe_shard_copy(ctx, 0, 0, torch.zeros(10, device="cuda"))
    with pytest.raises(ValueError, match="non-default stream"):
        from paper_2011_03479_gb300 import shard
        shard.GpuShard(rp, ci, 2, 0, 500, B.gempe_default_params(), stream=torch.cuda.default_stream())
