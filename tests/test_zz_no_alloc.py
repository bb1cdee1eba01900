"""The allocation-free slope fit, gempe_fit_sigma_static.

It exists for callers that must not allocate device memory where they call
the fit: code inside another allocator's callbacks, serving loops where
cudaMalloc/cudaFree would synchronise the device, and processes whose device
memory a framework has already reserved.  It stages the histogram in a static
device array instead of a per-call buffer, and must give the same sigma as
gempe_fit_sigma.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from conftest import gpu_available

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

TOL = 1e-4


def _histograms(seed, bins=1024):
    rng = np.random.default_rng(seed)
    he = np.zeros(bins); hn = np.zeros(bins)
    de = np.clip(rng.normal(rng.uniform(0.2, 1.8), 0.4, 4000), 0, 11.99)
    dn = np.clip(rng.normal(rng.uniform(1.5, 7.0), 1.2, 4000), 0, 11.99)
    np.add.at(he, (de / (12.0 / bins)).astype(int), 1.0)
    np.add.at(hn, (dn / (12.0 / bins)).astype(int), rng.uniform(5, 500))
    return he.astype(np.float32), hn.astype(np.float32)


def test_static_fit_matches_allocating_fit_twice():
    from paper_2011_03479_gb300 import binding as B
    lib = B.load()
    for seed in (1, 2):     # two calls in a row share (and overwrite) the static scratch
        he, hn = _histograms(seed)
        h = np.ascontiguousarray(np.concatenate([he, hn]), dtype=np.float32)
        out = ctypes.c_float()
        st = lib.gempe_fit_sigma_static(ctypes.c_void_p(h.ctypes.data), len(he), ctypes.c_float(12.0),
                                        ctypes.c_float(1.5), None, ctypes.byref(out))
        assert st == 0, B.gempe_last_error()
        ref = B.gempe_fit_sigma(he, hn)
        assert out.value == pytest.approx(ref, rel=TOL)


def test_static_fit_rejects_oversized_histograms():
    from paper_2011_03479_gb300 import binding as B
    he = np.zeros(4097, np.float32)
    with pytest.raises(B.GempeError) as err:
        B.gempe_fit_sigma_static(he, he)
    assert err.value.status == -1 and "4096" in str(err.value)
