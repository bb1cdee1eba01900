"""Failure detection on the device without a GPU fault: the tensor-core tile
kernel's bounded mbarrier wait is made to run out (a barrier phase nothing
completes, no MMA issued), and the give-up path must record GEMPE_E_TIMEOUT
for the host and free the CTA's TMEM; afterwards the device still runs the
tensor-core tiles of a BF16 block epoch within the parity bar."""
import numpy as np
import pytest

from conftest import gpu_available
from test_gpu_forms import TOL16, _bf16_errors, _run

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


def test_tile_wait_runs_out_and_reports_timeout(B, O, sbm_1000):
    for limit in (1, 64, 4096):
        status, freed = B.gempe_test_tile_wait(limit)
        assert status == -5, f"limit {limit}: status {status}"   # GEMPE_E_TIMEOUT
        assert freed == 1
    rp, ci = sbm_1000["row_ptr"], sbm_1000["col_idx"]
    x = (np.random.default_rng(164).normal(size=(1000, 64)) * 0.9).astype(np.float32)
    r = _run(B, O, rp, ci, 64, x, 0.8, 4, block_partners=64, precision=1)
    e_delta, e_z, e_x = _bf16_errors(r)
    assert e_delta.max() <= TOL16 and e_z.max() <= TOL16 and e_x.max() <= TOL16

