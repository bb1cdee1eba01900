"""GPU parity of Sec. III.F's second way to collect the slope histograms
(sigma_source = 1): after the update, a separate pass bins every edge and k
fresh samples per vertex at the new positions, and sigma is fitted on those.
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


@pytest.mark.parametrize("d", [2, 16])
def test_separate_pass_sigma_parity(B, O, sbm_1000, d):
    rp, ci = sbm_1000["row_ptr"], sbm_1000["col_idx"]
    x = (np.random.default_rng(90 + d).standard_normal((1000, d)) * 1.2).astype(np.float32)
    p = B.gempe_default_params(sigma_source=1, neg_per_vertex=6)
    with B.gempe_create(rp, ci, d, p) as ctx:
        B.gempe_set_positions(ctx, x)
        B.gempe_set_state(ctx, 0.9, 7)
        B.gempe_step(ctx, 1)
        s_gpu, e_gpu = B.gempe_get_state(ctx)
        xn = B.gempe_positions(ctx)
    ref = O.epoch(rp, ci, x.astype(np.float64), 0.9, 7, p.seed, 6)
    he, hn = O.hist_pass(rp, ci, ref["x_new"], 7, p.seed, 6)
    s_ref = O.sigma_fit(he, hn, 12.0, p.mu)
    assert e_gpu == 8
    assert s_gpu == pytest.approx(s_ref, rel=1e-4)
    err = np.abs(xn - ref["x_new"]).max() / np.abs(ref["x_new"]).max()
    assert err < 1e-4
    # the sweep's own histograms would give another slope: the source matters
    s_sweep = O.sigma_fit(ref["hist_e"], ref["hist_n"], 12.0, p.mu)
    assert abs(s_sweep - s_ref) > 1e-3 * s_ref


def test_separate_pass_full_run_loss(B, O, sbm_1000):
    rp, ci = sbm_1000["row_ptr"], sbm_1000["col_idx"]
    p = B.gempe_default_params(sigma_source=1)
    with B.gempe_create(rp, ci, 2, p) as ctx:
        x0 = B.gempe_positions(ctx)
        B.gempe_step(ctx, 200)
        x = B.gempe_positions(ctx)
        s, _ = B.gempe_get_state(ctx)
    xr, sr, _ = O.run(rp, ci, x0, 1.0, 200, p.seed, 5, sigma_source=1)
    pe_gpu = O.loss_sampled(rp, ci, x.astype(np.float64), s, 200, p.seed, 16)
    pe_ref = O.loss_sampled(rp, ci, xr, sr, 200, p.seed, 16)
    assert pe_gpu == pytest.approx(pe_ref, rel=0.01)
    assert s == pytest.approx(sr, rel=0.02)
