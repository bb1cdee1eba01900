import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


def bf16_round(x):
    """float32 values rounded to the nearest BF16 value (8 significant bits,
    ties to even), returned as float32: the rounding the BF16 form applies to
    the positions its pair arithmetic reads."""
    import numpy as np
    u = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).reshape(np.shape(x))


def gpu_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def sbm_small():
    """Two-block SBM with n=60 (tiny: brute force over all pairs is cheap)."""
    from paper_2011_03479_gb300 import inputs
    rp, ci = inputs.sbm([30, 30], 0.3, 0.03, seed=7)
    return rp, ci


@pytest.fixture(scope="session")
def sbm_1000():
    from paper_2011_03479_gb300 import inputs
    return inputs.sbm_1000()
