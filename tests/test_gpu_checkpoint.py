"""Checkpoint and resume (gempe_save / gempe_load).

A run of Fig. 4 stopped after some epochs and resumed from its checkpoint in
a new context continues as the uninterrupted run: the sampler statistics
exactly (the same samples: they are keyed by the graph and the epoch), the
positions and sigma up to the order of FP32 atomic additions (the bar of the
alone-vs-batch tests).  A checkpoint of another graph size, other sampling
parameters, a truncated or foreign buffer is refused and leaves the context
as it was.
"""
import numpy as np
import pytest

from conftest import gpu_available

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

INT_STATS = ("accepted", "rejected", "exhausted", "draws", "used", "epoch", "false_pos")


@pytest.fixture(scope="module")
def B():
    from paper_2011_03479_gb300 import binding
    binding.load()
    return binding


@pytest.mark.parametrize("form", [dict(neg_per_vertex=5), dict(neg_per_vertex=5, sampling=1),
                                  dict(block_partners=64, precision=1), dict(block_partners=64, precision=0),
                                  dict(neg_per_vertex=5, membership=1, rename_every=2),
                                  dict(neg_per_vertex=5, rng=1)],
                         ids=["per-vertex", "per-slot", "block-bf16", "block-fp32", "bytemap", "lcg"])
def test_resume_continues_the_run(B, sbm_1000, form):
    rp, ci = sbm_1000["row_ptr"], sbm_1000["col_idx"]
    d = 16 if form.get("block_partners") else 2
    p = B.gempe_default_params(**form)
    with B.gempe_create(rp, ci, d, p) as a:
        B.gempe_step(a, 3)
        blob = B.gempe_save(a)
        st_saved = B.gempe_stats(a)
        x_saved = B.gempe_positions(a)
        B.gempe_step(a, 4)
        x_a = B.gempe_positions(a)
        st_a = B.gempe_stats(a)
    assert len(blob) == 184 + 4 * x_saved.size
    with B.gempe_create(rp, ci, d, p) as b:
        B.gempe_load(b, blob)
        st_b0 = B.gempe_stats(b)
        for f in INT_STATS + ("sigma",):
            assert st_b0[f] == st_saved[f], f
        np.testing.assert_array_equal(B.gempe_positions(b), x_saved)
        B.gempe_step(b, 4)
        x_b = B.gempe_positions(b)
        st_b = B.gempe_stats(b)
    for f in INT_STATS:
        assert st_b[f] == st_a[f], f"{f}: {st_b[f]} != {st_a[f]}"
    tol = 1e-2 if form.get("precision") else 1e-3
    scale = max(float(np.abs(x_a).max()), 1e-30)
    err = float(np.abs(x_b.astype(np.float64) - x_a).max()) / scale
    assert err <= tol, f"positions differ by {err:.2e} of their scale"
    assert st_b["sigma"] == pytest.approx(st_a["sigma"], rel=tol)


def test_mismatched_checkpoint_refused(B, sbm_1000):
    rp, ci = sbm_1000["row_ptr"], sbm_1000["col_idx"]
    p = B.gempe_default_params(neg_per_vertex=5)
    with B.gempe_create(rp, ci, 2, p) as a:
        B.gempe_step(a, 2)
        blob = B.gempe_save(a)
    with B.gempe_create(rp, ci, 2, B.gempe_default_params(neg_per_vertex=5, seed=7)) as b:
        x0 = B.gempe_positions(b)
        s0 = B.gempe_get_state(b)
        with pytest.raises(B.GempeError, match="sampling parameters"):
            B.gempe_load(b, blob)
        with pytest.raises(B.GempeError, match="not a GEMPE checkpoint"):
            B.gempe_load(b, b"x" * len(blob))
        with pytest.raises(B.GempeError, match="too short"):
            B.gempe_load(b, blob[:100])
        np.testing.assert_array_equal(B.gempe_positions(b), x0)
        assert B.gempe_get_state(b) == s0
    with B.gempe_create(rp, ci, 2, p) as c:
        with pytest.raises(B.GempeError, match="truncated"):
            B.gempe_load(c, blob[:-4])
    with B.gempe_create(rp, ci, 4, p) as e:
        with pytest.raises(B.GempeError, match="another graph"):
            B.gempe_load(e, blob)
    with B.gempe_create(rp, ci, 2, B.gempe_default_params(neg_per_vertex=5, rng=1)) as g:
        with pytest.raises(B.GempeError, match="sampling parameters"):
            B.gempe_load(g, blob)
    for kw in (dict(mu=1.4), dict(hist_bins=512), dict(sigma_every=2), dict(w_formula=1), dict(clamp_neg_d=0)):
        with B.gempe_create(rp, ci, 2, B.gempe_default_params(neg_per_vertex=5, **kw)) as f:
            with pytest.raises(B.GempeError, match="another run"):
                B.gempe_load(f, blob)
