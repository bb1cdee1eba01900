"""The caller's device allocator (gempe_params.dev_alloc / dev_free).

A framework that owns the device memory hands its own allocator to the
engine; every device array of a context then comes from it and goes back to
it when the context is destroyed.  Checked with torch's caching allocator
behind the callbacks: an allocator that runs out (at the first, fourth or
ninth request) makes gempe_create fail with GEMPE_E_OOM and return every
block it had taken; the next context runs an epoch on the caller's blocks
and returns them all when it is destroyed.
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


class _Allocator:
    """torch's caching allocator behind the engine's callbacks, on one stream;
    fails every request from the `fail_at`-th on (0: never)."""

    def __init__(self, B, stream, fail_at=0):
        import torch
        self.live, self.n_alloc, self.n_free, self.fail_at = {}, 0, 0, fail_at

        def alloc(nbytes, user):
            if self.fail_at and self.n_alloc + 1 >= self.fail_at:
                return None
            ptr = torch.cuda.caching_allocator_alloc(nbytes, stream=stream)
            self.live[ptr] = nbytes
            self.n_alloc += 1
            return ptr

        def free(ptr, user):
            assert ptr in self.live, "a block the allocator did not hand out"
            torch.cuda.caching_allocator_delete(ptr)
            del self.live[ptr]
            self.n_free += 1

        self.alloc_fn, self.free_fn = B.ALLOC_FN(alloc), B.FREE_FN(free)


def test_caller_allocator_running_out(B, sbm_1000):
    import torch
    rp, ci = sbm_1000["row_ptr"], sbm_1000["col_idx"]
    s = torch.cuda.Stream()
    for fail_at in (1, 4, 9):
        al = _Allocator(B, s, fail_at=fail_at)
        p = B.gempe_default_params(block_partners=64, dev_alloc=al.alloc_fn, dev_free=al.free_fn)
        with pytest.raises(B.GempeError) as err:
            B.gempe_create(rp, ci, 64, p, stream=s)
        assert err.value.status == -3   # GEMPE_E_OOM
        assert al.n_alloc == fail_at - 1 and al.n_free == al.n_alloc and not al.live
    al = _Allocator(B, s)
    p = B.gempe_default_params(block_partners=64, dev_alloc=al.alloc_fn, dev_free=al.free_fn)
    with B.gempe_create(rp, ci, 64, p, stream=s) as ctx:
        B.gempe_step(ctx, 1)
        assert np.isfinite(B.gempe_positions(ctx)).all()
    assert al.n_free == al.n_alloc and not al.live
