"""Final-loss bar of the reduced-precision, batched and served forms: after a
full run, the predictive entropy (Eq. 2, sampled estimator) of the GPU's
final state is within 1% of the FP64 oracle's run from the same initial
positions and seed.  Both final states are scored by the oracle's own
estimator with the same loss samples, so only the trajectories differ.
"""
import numpy as np
import pytest

from conftest import gpu_available

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

SEED = 0x6E6D7065
LOSS_K = 32


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
def ba_4k():
    from paper_2011_03479_gb300 import inputs
    return inputs.barabasi_albert(4000, 8, seed=3201)


def _score(O, rp, ci, x, sigma, epochs, seed):
    return O.loss_sampled(rp, ci, np.asarray(x, np.float64), sigma, epochs, seed, LOSS_K)


def _oracle_final(O, rp, ci, d, epochs, seed, k, block=0):
    x0 = O.init_positions(len(rp) - 1, d, seed)
    xr, sr, _ = O.run(rp, ci, x0, 1.0, epochs, seed, k, block_partners=block)
    return _score(O, rp, ci, xr, sr, epochs, seed)


@pytest.mark.parametrize("precision", [1, 0])
def test_block_form_final_loss(B, O, ba_4k, precision):
    """Block sampling at d = 64: BF16 tensor-core tiles (precision 1) and the
    plain FP32 form (precision 0), 40 epochs."""
    rp, ci = ba_4k
    epochs = 40
    p = B.gempe_default_params(seed=SEED, block_partners=64, precision=precision)
    with B.gempe_create(rp, ci, 64, p) as ctx:
        B.gempe_step(ctx, epochs)
        x = B.gempe_positions(ctx)
        sigma, _ = B.gempe_get_state(ctx)
    pe_gpu = _score(O, rp, ci, x, sigma, epochs, SEED)
    pe_ref = _oracle_final(O, rp, ci, 64, epochs, SEED, 5, block=64)
    print(f"precision {precision}: PE gpu {pe_gpu:.6f} oracle {pe_ref:.6f}")
    assert pe_gpu == pytest.approx(pe_ref, rel=0.01)


def test_batched_form_final_loss(B, O):
    from paper_2011_03479_gb300 import inputs
    gs = inputs.sbm_batch(4, 300, 2500, dims=(2, 16, 64), seed=7100)
    epochs = 60
    p = B.gempe_default_params(seed=SEED, precision=1)
    with B.gempe_batch_create([(g["row_ptr"], g["col_idx"], g["d"]) for g in gs], p) as b:
        B.gempe_batch_step(b, epochs)
        finals = [(B.gempe_batch_positions(b, q), B.gempe_batch_stats(b, q)["sigma"]) for q in range(len(gs))]
    for q, (g, (x, s)) in enumerate(zip(gs, finals)):
        rp, ci = g["row_ptr"], g["col_idx"]
        pe_gpu = _score(O, rp, ci, x, s, epochs, SEED ^ q)
        pe_ref = _oracle_final(O, rp, ci, g["d"], epochs, SEED ^ q, 5)
        assert pe_gpu == pytest.approx(pe_ref, rel=0.01), f"graph {q} d={g['d']}"


@pytest.mark.parametrize("precision", [0, 1])
def test_served_form_final_loss(B, O, precision):
    """Served jobs (precision 1: BF16 positions for the d >= 8 jobs) against
    the FP64 oracle's runs of the same seeds."""
    from paper_2011_03479_gb300 import inputs
    jobs = []
    for q, (scale, d) in enumerate([(9, 2), (10, 32), (9, 128)]):
        rp, ci = inputs.rmat(scale, 10, seed=5301 + q)
        jobs.append((rp, ci, d, 0x5E5E1000 + q))
    epochs = 50
    p = B.gempe_default_params(neg_per_vertex=10, precision=precision)
    with B.gempe_server_create(4 << 30, max_jobs=4, params=p) as srv:
        ids = [B.gempe_server_submit(srv, rp, ci, d, epochs, s) for rp, ci, d, s in jobs]
        infos = [B.gempe_server_wait(srv, i, 120000) for i in ids]
        xs = [B.gempe_server_result(srv, i) for i in ids]
    for (rp, ci, d, s), inf, x in zip(jobs, infos, xs):
        pe_gpu = _score(O, rp, ci, x, inf["sigma"], epochs, s)
        pe_ref = _oracle_final(O, rp, ci, d, epochs, s, 10)
        assert pe_gpu == pytest.approx(pe_ref, rel=0.01), f"job d={d}"
