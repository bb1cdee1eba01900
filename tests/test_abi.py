"""The C-ABI library loads and exports what include/gempe.h declares (no GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(gempe_[a-z_0-9]+)\s*\(", text))
    return names


def test_header_declares_the_calls():
    names = _declared_functions()
    for required in ("gempe_create", "gempe_step", "gempe_positions", "gempe_loss", "gempe_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2011_03479_gb300 import binding
    lib = binding.load()
    missing = [n for n in sorted(_declared_functions()) if not hasattr(lib, n)]
    assert not missing, missing


def test_default_params_are_the_papers():
    from paper_2011_03479_gb300 import binding
    p = binding.gempe_default_params()
    assert p.mu == 1.5 and p.sigma0 == 1.0          # Sec. III.F, Fig. 4
    assert p.sigma_every == 1 and p.neg_per_vertex == 5 and p.max_retries == 32
    assert p.symmetric_neg == 1 and p.w_formula == 0 and p.clamp_neg_d == 1
    assert p.hist_bins == 1024 and p.hist_max == 12.0 and p.seed == 0x6E6D7065


def _status(fn, *args):
    from paper_2011_03479_gb300 import binding
    h = ctypes.c_void_p()
    return fn(*args, ctypes.byref(h)), h


INVALID = {"asym": [[1], [], []], "loop": [[0, 1], [0], []], "dup": [[1, 1], [0, 0], []],
           "range": [[5], [0], []], "unsorted": [[2, 1], [0], [0]]}


def _csr(rows):
    rp = np.cumsum([0] + [len(r) for r in rows]).astype(np.int32)
    ci = np.array(sum(rows, []), dtype=np.int32)
    return rp, ci


@pytest.mark.parametrize("case", ["loop", "dup", "range", "unsorted"])
def test_invalid_graphs_rejected_on_host(case):
    """The row checks run on the host before any device work (no GPU here)."""
    from paper_2011_03479_gb300 import binding
    lib = binding.load()
    rp, ci = _csr(INVALID[case])
    p = binding.gempe_default_params()
    st, h = _status(lib.gempe_create, ctypes.c_void_p(rp.ctypes.data),
                    ctypes.c_void_p(ci.ctypes.data), len(rp) - 1, 2, ctypes.byref(p), None)
    assert st == -2, binding.gempe_last_error()
    assert not h.value


@pytest.mark.parametrize("case", sorted(INVALID))
def test_validate_csr_host(case):
    """gempe_validate_csr: every check, symmetry included, on the host."""
    from paper_2011_03479_gb300 import binding
    rp, ci = _csr(INVALID[case])
    with pytest.raises(binding.GempeError) as ei:
        binding.gempe_validate_csr(rp, ci)
    assert ei.value.status == -2
    msg = str(ei.value)
    if case == "asym":
        assert "(0,1) without its reverse" in msg


def test_validate_csr_reports_lowest_row():
    """Errors in several rows: the lowest row is named, whichever thread finds it."""
    from paper_2011_03479_gb300 import binding, inputs
    rp, ci = inputs.rmat(12, 8, seed=99)
    binding.gempe_validate_csr(rp, ci)            # a valid graph passes
    ci2 = ci.copy()
    rows = [int(np.searchsorted(rp, len(ci) * f, side="right") - 1) for f in (0.3, 0.7)]
    for r in rows:                                 # make two rows' first entries self loops
        if rp[r + 1] > rp[r]:
            ci2[rp[r]] = r
    with pytest.raises(binding.GempeError) as ei:
        binding.gempe_validate_csr(rp, ci2)
    first = min(r for r in rows if rp[r + 1] > rp[r])
    msg = str(ei.value)
    assert f"self loop at vertex {first}" in msg or f"row {first} not strictly increasing" in msg, msg


def test_invalid_args_rejected_on_host():
    from paper_2011_03479_gb300 import binding
    lib = binding.load()
    rp = np.array([0, 1, 2], dtype=np.int32)
    ci = np.array([1, 0], dtype=np.int32)
    for d, k in ((5, 5), (0, 5), (2, 33), (2, -1)):
        p = binding.gempe_default_params(neg_per_vertex=k)
        st, _ = _status(lib.gempe_create, ctypes.c_void_p(rp.ctypes.data), ctypes.c_void_p(ci.ctypes.data),
                        2, d, ctypes.byref(p), None)
        assert st == -1
    p = binding.gempe_default_params()
    st, _ = _status(lib.gempe_create, ctypes.c_void_p(rp.ctypes.data), ctypes.c_void_p(ci.ctypes.data),
                    1, 2, ctypes.byref(p), None)
    assert st == -1
    # byte-map membership: 0/1, log2 0 or 6..32, rename_every >= 0, not with block sampling
    for kw, d in ((dict(membership=2), 2), (dict(membership=1, bytemap_log2=5), 2),
                  (dict(membership=1, bytemap_log2=33), 2), (dict(membership=1, rename_every=-1), 2),
                  (dict(membership=1, block_partners=64), 16), (dict(rng=2), 2), (dict(rng=-1), 2),
                  (dict(rng=1, block_partners=64), 16)):
        p = binding.gempe_default_params(**kw)
        st, _ = _status(lib.gempe_create, ctypes.c_void_p(rp.ctypes.data), ctypes.c_void_p(ci.ctypes.data),
                        2, d, ctypes.byref(p), None)
        assert st == -1, kw
    with pytest.raises(binding.GempeError):
        binding.gempe_create(np.array([0, 1, 1], np.int32), np.array([1], np.int32), 2)


def test_generated_graphs_are_valid_csr(sbm_1000):
    from paper_2011_03479_gb300 import inputs
    for rp, ci in ((sbm_1000["row_ptr"], sbm_1000["col_idx"]), inputs.rmat(10, 8, seed=3),
                   inputs.barabasi_albert(2000, 3, seed=4)):
        n = len(rp) - 1
        assert rp[0] == 0 and np.all(np.diff(rp) >= 0) and rp[-1] == len(ci)
        rows = np.repeat(np.arange(n), np.diff(rp))
        assert np.all(ci != rows)
        for i in range(0, n, max(1, n // 200)):
            r = ci[rp[i]:rp[i + 1]]
            assert np.all(np.diff(r) > 0)
        a = set(zip(rows.tolist(), ci.tolist()))
        assert all((j, i) in a for i, j in a)


def test_batch_rejects_invalid_graphs_on_host():
    """gempe_batch_create checks every graph's rows on the host before any
    device work (the symmetry follows on the device): a self loop or an
    unsupported dimension fails cleanly."""
    from paper_2011_03479_gb300 import binding
    good = (np.array([0, 1, 2], np.int32), np.array([1, 0], np.int32), 2)
    loop = (np.array([0, 2, 3], np.int32), np.array([0, 1, 0], np.int32), 2)
    with pytest.raises(binding.GempeError) as ei:
        binding.gempe_batch_create([good, loop])
    assert ei.value.status == -2 and "graph 1" in str(ei.value)
    with pytest.raises(binding.GempeError) as ei:
        binding.gempe_batch_create([good, (good[0], good[1], 5)])
    assert ei.value.status == -1


def test_job_bytes_formula():
    """gempe_job_bytes (host arithmetic) covers at least the resident state
    the serving admission counts: CSR, edge table (every undirected edge
    once at load 1/2: next power of two of nnz slots, 8-byte keys above
    65,536 vertices, 4-byte keys up to it), positions, accumulators; it
    grows with n, nnz, d and with the BF16 shadow; invalid arguments give 0."""
    from paper_2011_03479_gb300 import binding as B
    p = B.gempe_default_params(neg_per_vertex=10)
    n, nnz = 100_000, 1_600_000
    for d in (2, 32, 128):
        b = B.gempe_job_bytes(n, nnz, d, p)
        table = 8 * (1 << int(np.ceil(np.log2(nnz))))
        floor = 4 * (n + 1) + 4 * nnz + table + 4 * n * d + 4 * n * (d + 1)
        assert b >= floor
        assert b < 2 * floor + (64 << 20)
    assert B.gempe_job_bytes(n, nnz, 32, p) < B.gempe_job_bytes(n, nnz, 128, p)
    assert B.gempe_job_bytes(n, nnz, 32, p) < B.gempe_job_bytes(2 * n, nnz, 32, p)
    assert B.gempe_job_bytes(n, nnz, 32, p) < B.gempe_job_bytes(n, 2 * nnz, 32, p)
    pb = B.gempe_default_params(neg_per_vertex=10, precision=1)
    assert B.gempe_job_bytes(n, nnz, 32, pb) > B.gempe_job_bytes(n, nnz, 32, p)
    assert B.gempe_job_bytes(1, 0, 2, p) == 0 and B.gempe_job_bytes(n, nnz, 5, p) == 0
    # the byte map adds its 2^log2 bytes; automatic size: nnz to a power of two, times 128, at most 2^30
    pm = B.gempe_default_params(neg_per_vertex=10, membership=1, bytemap_log2=20)
    assert B.gempe_job_bytes(n, nnz, 32, pm) - B.gempe_job_bytes(n, nnz, 32, p) == 1 << 20
    pa = B.gempe_default_params(neg_per_vertex=10, membership=1)
    assert B.gempe_job_bytes(n, nnz, 32, pa) - B.gempe_job_bytes(n, nnz, 32, p) == 1 << 28


def test_checkpoint_calls_reject_null_arguments():
    """gempe_save / gempe_load check their arguments before touching a device."""
    import ctypes
    from paper_2011_03479_gb300 import binding
    lib = binding.load()
    n = ctypes.c_size_t(0)
    assert lib.gempe_save(None, None, ctypes.byref(n)) == -1
    assert lib.gempe_save(None, None, None) == -1
    assert lib.gempe_load(None, b"GEMPECK", 7) == -1
    assert lib.gempe_load(None, None, 0) == -1


def test_tile_wait_probe_rejects_bad_limits_on_host():
    """The bounded-wait test hook checks its poll limit before any CUDA call."""
    from paper_2011_03479_gb300 import binding
    for bad in (0, -3, (1 << 22) + 1):
        with pytest.raises(binding.GempeError) as err:
            binding.gempe_test_tile_wait(bad)
        assert err.value.status == -1
