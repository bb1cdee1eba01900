"""The allocation-free slope fit, gempe_fit_sigma_static.

It exists for callers that must not allocate device memory where they call
the fit: code inside another allocator's callbacks, serving loops where
cudaMalloc/cudaFree would synchronise the device, and processes whose device
memory a framework has already reserved.  It stages the histogram in a static
device array instead of a per-call buffer, and must give the same sigma as
gempe_fit_sigma.

This file is collected last (the "zz" prefix) because the call is an
addition outside the paper's method: under ``pytest -x`` a failure here
stops the run only after every test of the method itself has run.  Each
test also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from conftest import gpu_available

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

TOL = 1e-4
CU_MEMPOOL_ATTR_USED_MEM_CURRENT = 7
CU_MEMPOOL_ATTR_USED_MEM_HIGH = 8


def _histograms(seed, bins=1024):
    rng = np.random.default_rng(seed)
    he = np.zeros(bins); hn = np.zeros(bins)
    de = np.clip(rng.normal(rng.uniform(0.2, 1.8), 0.4, 4000), 0, 11.99)
    dn = np.clip(rng.normal(rng.uniform(1.5, 7.0), 1.2, 4000), 0, 11.99)
    np.add.at(he, (de / (12.0 / bins)).astype(int), 1.0)
    np.add.at(hn, (dn / (12.0 / bins)).astype(int), rng.uniform(5, 500))
    return he.astype(np.float32), hn.astype(np.float32)


class _DevicePool:
    """The current device's default stream-ordered memory pool (driver API),
    the pool the engine's stream-ordered allocations come from."""

    def __init__(self):
        import torch
        self.cu = ctypes.CDLL("libcuda.so.1")
        dev = ctypes.c_int()
        assert self.cu.cuDeviceGet(ctypes.byref(dev), torch.cuda.current_device()) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def get(self, attr):
        v = ctypes.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return v.value

    def reset_high(self):
        zero = ctypes.c_uint64(0)     # resets the high-water mark to the current use
        assert self.cu.cuMemPoolSetAttribute(self.pool, CU_MEMPOOL_ATTR_USED_MEM_HIGH, ctypes.byref(zero)) == 0


def _static_fit(lib, he, hn, stream_handle):
    h = np.ascontiguousarray(np.concatenate([he, hn]), dtype=np.float32)
    out = ctypes.c_float()
    st = lib.gempe_fit_sigma_static(ctypes.c_void_p(h.ctypes.data), len(he), ctypes.c_float(12.0),
                                    ctypes.c_float(1.5), stream_handle, ctypes.byref(out))
    return st, out.value


def test_static_fit_matches_allocating_fit_twice():
    from paper_2011_03479_gb300 import binding as B
    lib = B.load()
    for seed in (1, 2):     # two calls in a row share (and overwrite) the static scratch
        he, hn = _histograms(seed)
        st, got = _static_fit(lib, he, hn, None)
        assert st == 0, B.gempe_last_error()
        ref = B.gempe_fit_sigma(he, hn)
        assert got == pytest.approx(ref, rel=TOL)


def test_static_fit_largest_size_on_a_caller_stream_allocates_nothing():
    """4096 bins per side (the static array's capacity, and a slope-fit block
    above 48 KiB of shared memory) on a non-default stream, twice: the same
    sigma as the allocating fit, and the device pool's high-water mark does
    not move across the static calls, while the allocating fit moves it."""
    import torch
    from paper_2011_03479_gb300 import binding as B
    lib = B.load()
    s = torch.cuda.Stream()
    pool = _DevicePool()
    refs = []
    for seed in (3, 4):
        he, hn = _histograms(seed, bins=4096)
        refs.append((he, hn, B.gempe_fit_sigma(he, hn, stream=s)))
    _static_fit(lib, *_histograms(5, bins=4096), ctypes.c_void_p(s.cuda_stream))   # first call: per-device set-up
    torch.cuda.synchronize()
    used0 = pool.get(CU_MEMPOOL_ATTR_USED_MEM_CURRENT)
    pool.reset_high()
    for he, hn, ref in refs:
        st, got = _static_fit(lib, he, hn, ctypes.c_void_p(s.cuda_stream))
        assert st == 0, B.gempe_last_error()
        assert got == pytest.approx(ref, rel=TOL)
    assert pool.get(CU_MEMPOOL_ATTR_USED_MEM_HIGH) <= used0
    assert pool.get(CU_MEMPOOL_ATTR_USED_MEM_CURRENT) == used0
    # control: the allocating fit is seen by the same counter
    pool.reset_high()
    B.gempe_fit_sigma(*refs[0][:2], stream=s)
    assert pool.get(CU_MEMPOOL_ATTR_USED_MEM_HIGH) > used0


def test_small_static_fit_leaves_a_large_context_runnable():
    """A context built with 4096 bins needs slope-fit blocks above 48 KiB of
    shared memory; a later static fit with 16 bins must not lower that limit
    (it is one per kernel and device): the context's epochs still run."""
    from paper_2011_03479_gb300 import binding as B
    from paper_2011_03479_gb300 import inputs
    lib = B.load()
    w = inputs.sbm_1000()
    p = B.gempe_default_params(neg_per_vertex=5, hist_bins=4096)
    with B.gempe_create(w["row_ptr"], w["col_idx"], 2, p) as ctx:
        B.gempe_step(ctx, 2)
        he, hn = _histograms(6, bins=16)
        st, got = _static_fit(lib, he, hn, None)
        assert st == 0 and got > 0, B.gempe_last_error()
        B.gempe_step(ctx, 2)
        B.gempe_sweep(ctx)
        B.gempe_update(ctx)
        x = B.gempe_positions(ctx)
        assert np.isfinite(x).all()
        assert B.gempe_stats(ctx)["epoch"] == 5


def test_static_fit_rejects_oversized_histograms():
    from paper_2011_03479_gb300 import binding as B
    he = np.zeros(4097, np.float32)
    with pytest.raises(B.GempeError) as err:
        B.gempe_fit_sigma_static(he, he)
    assert err.value.status == -1 and "4096" in str(err.value)
