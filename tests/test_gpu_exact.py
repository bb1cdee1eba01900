"""GPU parity of the exact predictive entropy (Eq. 2 over all pairs) and of
its minimum over the slope, against the FP64 oracle's brute force.

Bars: the exact sum within 1e-5 relative (FP32 pair terms, FP64 sums, as
for the sampled loss); the minimising slope within 1e-4 relative of the
oracle's bisection on the exact derivative.
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


def _graphs():
    from paper_2011_03479_gb300 import inputs
    return {
        "sbm-1000": inputs.sbm([250, 250, 250, 250], 0.05, 0.002, seed=1001),
        "rmat-s10": inputs.rmat(10, 8, seed=6001),                  # isolated vertices, n multiple of 64
        "sbm-ragged": inputs.sbm([301, 180, 250], 0.04, 0.003, seed=6002),   # n = 731, ragged last tile
        "pair": (np.array([0, 1, 2], np.int32), np.array([1, 0], np.int32)),
    }


GRAPHS = _graphs()


@pytest.mark.parametrize("name,d", [("sbm-1000", 2), ("sbm-1000", 16), ("rmat-s10", 3), ("sbm-ragged", 64),
                                    ("sbm-ragged", 256), ("pair", 2), ("rmat-s10", 1)])
def test_exact_loss_parity(B, O, name, d):
    rp, ci = GRAPHS[name]
    n = len(rp) - 1
    x = (np.random.default_rng(d + n).normal(size=(n, d)) * 1.3).astype(np.float32)
    sigma = 0.8
    with B.gempe_create(rp, ci, d, B.gempe_default_params()) as ctx:
        B.gempe_set_positions(ctx, x)
        B.gempe_set_state(ctx, sigma, 0)
        pe, s = B.gempe_loss_exact(ctx)
    assert s == pytest.approx(sigma)
    ref = O.loss_exact(rp, ci, x.astype(np.float64), sigma)
    assert pe == pytest.approx(ref, rel=1e-5)


@pytest.mark.parametrize("name,d", [("sbm-1000", 2), ("sbm-ragged", 16), ("rmat-s10", 2)])
def test_exact_sigma_minimum_parity(B, O, name, d):
    rp, ci = GRAPHS[name]
    n = len(rp) - 1
    x = (np.random.default_rng(7 * d + n).normal(size=(n, d)) * 1.1).astype(np.float32)
    with B.gempe_create(rp, ci, d, B.gempe_default_params()) as ctx:
        B.gempe_set_positions(ctx, x)
        B.gempe_set_state(ctx, 0.5, 0)
        pe, s = B.gempe_loss_exact(ctx, fit_sigma=True)
        assert B.gempe_get_state(ctx)[0] == pytest.approx(0.5)      # the context's slope is untouched
    xs = x.astype(np.float64)
    s_ref = O.sigma_fit_exact(rp, ci, xs)
    assert s == pytest.approx(s_ref, rel=1e-4)
    assert pe == pytest.approx(O.loss_exact(rp, ci, xs, s_ref), rel=1e-5)


def test_exact_minimum_after_training(B, O):
    """After 100 epochs of the SBM drawing the exact minimum over sigma is no
    larger than the exact entropy at the slope the histograms gave."""
    rp, ci = GRAPHS["sbm-1000"]
    with B.gempe_create(rp, ci, 2, B.gempe_default_params()) as ctx:
        B.gempe_step(ctx, 100)
        pe_hist, s_hist = B.gempe_loss_exact(ctx)
        pe_min, s_min = B.gempe_loss_exact(ctx, fit_sigma=True)
        x = B.gempe_positions(ctx)
    assert pe_min <= pe_hist * (1 + 1e-6)
    assert s_min == pytest.approx(O.sigma_fit_exact(rp, ci, x.astype(np.float64)), rel=1e-4)
    # the histogram slope (1024 bins) is close to the exact one
    assert s_hist == pytest.approx(s_min, rel=0.05)
