"""ctypes binding of the C ABI in ``include/gempe.h``.

Argument marshalling only: every step of the epoch runs in ``libgempe.so``'s
CUDA kernels.  The functions keep the C names.  Host arrays are numpy arrays;
device arrays may be torch CUDA tensors (their ``data_ptr()`` is passed) and a
``stream`` argument may be a ``torch.cuda.Stream`` or a raw ``cudaStream_t``.

Importing this module does not need a GPU; loading the library does not
either.  If the library cannot be built or loaded the import fails: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

GEMPE_OK = 0
STATUS_NAMES = {0: "GEMPE_OK", -1: "GEMPE_E_INVALID_ARG", -2: "GEMPE_E_INVALID_GRAPH",
                -3: "GEMPE_E_OOM", -4: "GEMPE_E_CUDA", -5: "GEMPE_E_TIMEOUT",
                -6: "GEMPE_E_NUMERIC", -7: "GEMPE_E_BUDGET"}

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class gempe_params(ctypes.Structure):
    _fields_ = [
        ("mu", ctypes.c_float),
        ("sigma0", ctypes.c_float),
        ("sigma_every", ctypes.c_int32),
        ("neg_per_vertex", ctypes.c_int32),
        ("max_retries", ctypes.c_int32),
        ("symmetric_neg", ctypes.c_int32),
        ("w_formula", ctypes.c_int32),
        ("clamp_neg_d", ctypes.c_int32),
        ("z_min", ctypes.c_float),
        ("init_range", ctypes.c_float),
        ("seed", ctypes.c_uint64),
        ("hist_bins", ctypes.c_int32),
        ("hist_max", ctypes.c_float),
        ("precision", ctypes.c_int32),
        ("block_partners", ctypes.c_int32),
        ("tile_vertices", ctypes.c_int32),
        ("sampling", ctypes.c_int32),
        ("sigma_source", ctypes.c_int32),
        ("autotune", ctypes.c_int32),
        ("membership", ctypes.c_int32),
        ("bytemap_log2", ctypes.c_int32),
        ("rename_every", ctypes.c_int32),
        ("rng", ctypes.c_int32),
        ("dev_alloc", ALLOC_FN),
        ("dev_free", FREE_FN),
        ("alloc_user", ctypes.c_void_p),
    ]


class gempe_stats_t(ctypes.Structure):
    _fields_ = [
        ("epoch", ctypes.c_int32),
        ("sigma", ctypes.c_float),
        ("accepted", ctypes.c_uint64),
        ("rejected", ctypes.c_uint64),
        ("exhausted", ctypes.c_uint64),
        ("draws", ctypes.c_uint64),
        ("used", ctypes.c_uint64),
        ("n_edges", ctypes.c_int64),
        ("n", ctypes.c_int32),
        ("d", ctypes.c_int32),
        ("k", ctypes.c_int32),
        ("sigma_iters", ctypes.c_int32),
        ("false_pos", ctypes.c_uint64),
    ]


class gempe_graph_desc(ctypes.Structure):
    _fields_ = [
        ("row_ptr", ctypes.c_void_p),
        ("col_idx", ctypes.c_void_p),
        ("n", ctypes.c_int32),
        ("d", ctypes.c_int32),
    ]


class gempe_job_desc(ctypes.Structure):
    _fields_ = [
        ("row_ptr", ctypes.c_void_p),
        ("col_idx", ctypes.c_void_p),
        ("n", ctypes.c_int32),
        ("d", ctypes.c_int32),
        ("epochs", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
    ]


class gempe_job_info(ctypes.Structure):
    _fields_ = [
        ("state", ctypes.c_int32),
        ("epochs", ctypes.c_int32),
        ("epochs_done", ctypes.c_int32),
        ("submit_ns", ctypes.c_uint64),
        ("admit_ns", ctypes.c_uint64),
        ("done_ns", ctypes.c_uint64),
        ("device_bytes", ctypes.c_uint64),
        ("pairs", ctypes.c_uint64),
        ("sigma", ctypes.c_float),
    ]


class GempeError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lib = None


def library_path() -> str:
    return _build.GEMPE_LIB


def load(build: bool = True):
    """Load libgempe.so (building it first when missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build_gempe() if build else _build.GEMPE_LIB
    if not os.path.exists(path):
        raise RuntimeError(f"GEMPE CUDA engine not found at {path}; run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
    st = ctypes.c_int
    sig = {
        "gempe_default_params": (None, [P(gempe_params)]),
        "gempe_validate_csr": (st, [vp, vp, i32]),
        "gempe_create": (st, [vp, vp, i32, i32, P(gempe_params), vp, P(vp)]),
        "gempe_create_device": (st, [vp, vp, i32, i64, i32, P(gempe_params), vp, P(vp)]),
        "gempe_destroy": (None, [vp]),
        "gempe_step": (st, [vp, i32]),
        "gempe_sweep": (st, [vp, vp]),
        "gempe_update": (st, [vp]),
        "gempe_positions": (st, [vp, vp, sz]),
        "gempe_positions_device": (st, [vp, P(vp)]),
        "gempe_set_positions": (st, [vp, vp, sz]),
        "gempe_set_state": (st, [vp, ctypes.c_float, i32]),
        "gempe_get_state": (st, [vp, P(ctypes.c_float), P(i32)]),
        "gempe_accumulators": (st, [vp, vp, sz]),
        "gempe_histograms": (st, [vp, vp, sz]),
        "gempe_sample": (st, [vp, i32, vp, sz]),
        "gempe_is_edge": (st, [vp, vp, sz, vp]),
        "gempe_loss": (st, [vp, P(ctypes.c_double), P(ctypes.c_float)]),
        "gempe_loss_exact": (st, [vp, i32, P(ctypes.c_double), P(ctypes.c_float)]),
        "gempe_fit_sigma": (st, [vp, i32, ctypes.c_float, ctypes.c_float, vp, P(ctypes.c_float)]),
        "gempe_fit_sigma_static": (st, [vp, i32, ctypes.c_float, ctypes.c_float, vp, P(ctypes.c_float)]),
        "gempe_test_tile_wait": (st, [i32, P(i32), P(i32)]),
        "gempe_kernel_times": (st, [vp, i32, P(ctypes.c_float)]),
        "gempe_create_shard": (st, [vp, vp, i32, i32, i32, i32, P(gempe_params), vp, P(vp)]),
        "gempe_shard_layout": (st, [vp, P(i64)]),
        "gempe_shard_copy": (st, [vp, i32, i32, vp]),
        "gempe_stats": (st, [vp, P(gempe_stats_t)]),
        "gempe_save": (st, [vp, vp, P(sz)]),
        "gempe_load": (st, [vp, vp, sz]),
        "gempe_set_shape": (st, [vp, P(i32)]),
        "gempe_get_shape": (st, [vp, P(i32)]),
        "gempe_last_error": (ctypes.c_char_p, []),
        "gempe_batch_create": (st, [i32, P(gempe_graph_desc), P(gempe_params), vp, P(vp)]),
        "gempe_batch_destroy": (None, [vp]),
        "gempe_batch_step": (st, [vp, i32]),
        "gempe_batch_positions": (st, [vp, i32, vp, sz]),
        "gempe_batch_loss": (st, [vp, i32, P(ctypes.c_double), P(ctypes.c_float)]),
        "gempe_batch_stats": (st, [vp, i32, P(gempe_stats_t)]),
        "gempe_batch_shape": (st, [vp, i32, P(i64)]),
        "gempe_job_bytes": (sz, [i32, i64, i32, P(gempe_params)]),
        "gempe_server_create": (st, [sz, i32, P(gempe_params), P(vp)]),
        "gempe_server_destroy": (None, [vp]),
        "gempe_server_submit": (st, [vp, P(gempe_job_desc), P(ctypes.c_uint64)]),
        "gempe_server_poll": (st, [vp, ctypes.c_uint64, P(gempe_job_info)]),
        "gempe_server_wait": (st, [vp, ctypes.c_uint64, i32, P(gempe_job_info)]),
        "gempe_server_result": (st, [vp, ctypes.c_uint64, vp, sz]),
        "gempe_server_stats": (st, [vp, P(i64)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(status: int) -> None:
    if status != GEMPE_OK:
        msg = load().gempe_last_error()
        raise GempeError(status, msg.decode() if msg else "")


def _stream_handle(stream) -> ctypes.c_void_p:
    if stream is None:
        return ctypes.c_void_p(None)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _ptr(a: np.ndarray) -> ctypes.c_void_p:
    return ctypes.c_void_p(a.ctypes.data)


# ---------------------------------------------------------------------------
# The C calls, same names
# ---------------------------------------------------------------------------
def gempe_default_params(**overrides) -> gempe_params:
    p = gempe_params()
    load().gempe_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


class _Ctx:
    """Owned context handle (destroyed with gempe_destroy on close / GC)."""

    def __init__(self, handle, n, d, k, keep=(), slots=None, per_slot=False, nnz=0):
        self.handle = handle
        self.n, self.d, self.k = n, d, k
        self.slots = k if slots is None else slots   # sample slots per vertex in a sweep
        self.per_slot, self.nnz = per_slot, nnz      # Sec. III.C's policy: one sample per CSR slot
        self._keep = keep   # allocator callbacks must outlive the context

    def close(self):
        if self.handle:
            load().gempe_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def gempe_create(row_ptr, col_idx, d: int, params: gempe_params | None = None, stream=None) -> _Ctx:
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    n = len(rp) - 1
    p = params or gempe_default_params()
    h = ctypes.c_void_p()
    _check(load().gempe_create(_ptr(rp), _ptr(ci) if len(ci) else ctypes.c_void_p(None), n, d,
                               ctypes.byref(p), _stream_handle(stream), ctypes.byref(h)))
    return _Ctx(h, n, d, p.neg_per_vertex, keep=(p,), slots=p.block_partners or p.neg_per_vertex,
                per_slot=(p.sampling == 1), nnz=len(ci))


def gempe_create_shard(row_ptr, col_idx, d: int, v_begin: int, v_end: int, params: gempe_params | None = None,
                       stream=None) -> _Ctx:
    """A shard of one graph: anchors v_begin <= i < v_end (see shard.py)."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    n = len(rp) - 1
    p = params or gempe_default_params()
    h = ctypes.c_void_p()
    _check(load().gempe_create_shard(_ptr(rp), _ptr(ci) if len(ci) else ctypes.c_void_p(None), n, d, int(v_begin),
                                     int(v_end), ctypes.byref(p), _stream_handle(stream), ctypes.byref(h)))
    return _Ctx(h, n, d, p.neg_per_vertex, keep=(p,), slots=p.block_partners or p.neg_per_vertex,
                per_slot=(p.sampling == 1), nnz=len(ci))


SHARD_SUMS, SHARD_HIST_E, SHARD_HIST_C, SHARD_HIST_D, SHARD_HIST_X, SHARD_POSITIONS = range(6)


def gempe_shard_layout(ctx: _Ctx) -> dict:
    out = (ctypes.c_int64 * 4)()
    _check(load().gempe_shard_layout(ctx.handle, out))
    return {"sum_floats": int(out[0]), "stride": int(out[1]), "bins": int(out[2]), "position_floats": int(out[3])}


def gempe_shard_copy(ctx: _Ctx, what: int, direction: int, device_buf) -> None:
    """direction 0: the context's array `what` into device_buf (a CUDA tensor
    or a device address); 1: device_buf into the context."""
    ptr = device_buf.data_ptr() if hasattr(device_buf, "data_ptr") else int(device_buf)
    _check(load().gempe_shard_copy(ctx.handle, int(what), int(direction), ctypes.c_void_p(ptr)))


def gempe_create_device(d_row_ptr, d_col_idx, d: int, params: gempe_params | None = None,
                        stream=None) -> _Ctx:
    """CSR given as torch CUDA int32 tensors."""
    n = d_row_ptr.numel() - 1
    nnz = d_col_idx.numel()
    p = params or gempe_default_params()
    h = ctypes.c_void_p()
    _check(load().gempe_create_device(ctypes.c_void_p(d_row_ptr.data_ptr()),
                                      ctypes.c_void_p(d_col_idx.data_ptr() if nnz else None), n, nnz, d,
                                      ctypes.byref(p), _stream_handle(stream), ctypes.byref(h)))
    return _Ctx(h, n, d, p.neg_per_vertex, keep=(p,), slots=p.block_partners or p.neg_per_vertex,
                per_slot=(p.sampling == 1), nnz=nnz)


def gempe_destroy(ctx: _Ctx) -> None:
    ctx.close()


def gempe_validate_csr(row_ptr, col_idx) -> None:
    """Host-only check of a CSR graph (raises GempeError when it is invalid)."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    _check(load().gempe_validate_csr(_ptr(rp), _ptr(ci) if ci.size else None, len(rp) - 1))


def gempe_step(ctx: _Ctx, iters: int = 1) -> None:
    _check(load().gempe_step(ctx.handle, int(iters)))


def gempe_sweep(ctx: _Ctx, record_samples: bool = False):
    slots = ctx.slots
    if record_samples and ctx.per_slot:
        out = np.empty(max(ctx.nnz, 1), dtype=np.int32)
        _check(load().gempe_sweep(ctx.handle, _ptr(out)))
        return out[: ctx.nnz]
    if record_samples and slots > 0:
        out = np.empty(ctx.n * slots, dtype=np.int32)
        _check(load().gempe_sweep(ctx.handle, _ptr(out)))
        return out.reshape(ctx.n, slots)
    _check(load().gempe_sweep(ctx.handle, ctypes.c_void_p(None)))
    return None


def gempe_update(ctx: _Ctx) -> None:
    _check(load().gempe_update(ctx.handle))


def gempe_positions(ctx: _Ctx, out: np.ndarray | None = None) -> np.ndarray:
    if out is None:
        out = np.empty((ctx.n, ctx.d), dtype=np.float32)
    assert out.dtype == np.float32 and out.flags.c_contiguous and out.size == ctx.n * ctx.d
    _check(load().gempe_positions(ctx.handle, _ptr(out), out.size))
    return out


def gempe_positions_device(ctx: _Ctx) -> int:
    v = ctypes.c_void_p()
    _check(load().gempe_positions_device(ctx.handle, ctypes.byref(v)))
    return v.value


def gempe_set_positions(ctx: _Ctx, x) -> None:
    x = np.ascontiguousarray(x, dtype=np.float32)
    _check(load().gempe_set_positions(ctx.handle, _ptr(x), x.size))


def gempe_set_state(ctx: _Ctx, sigma: float, epoch: int) -> None:
    _check(load().gempe_set_state(ctx.handle, float(sigma), int(epoch)))


def gempe_get_state(ctx: _Ctx):
    s = ctypes.c_float()
    e = ctypes.c_int32()
    _check(load().gempe_get_state(ctx.handle, ctypes.byref(s), ctypes.byref(e)))
    return s.value, e.value


def gempe_save(ctx: _Ctx) -> bytes:
    """Checkpoint of the context between epochs (positions, sigma, epoch, sampler statistics)."""
    n = ctypes.c_size_t(0)
    _check(load().gempe_save(ctx.handle, None, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value)
    _check(load().gempe_save(ctx.handle, buf, ctypes.byref(n)))
    return buf.raw[: n.value]


def gempe_load(ctx: _Ctx, data: bytes) -> None:
    """Resume the context from a gempe_save checkpoint of the same graph and sampling parameters."""
    b = bytes(data)
    _check(load().gempe_load(ctx.handle, b, len(b)))


def gempe_accumulators(ctx: _Ctx):
    """Returns (delta, z): delta[i] = y_i - z_i x_i (Eq. 3), z[i] = z_i."""
    out = np.empty((ctx.n, ctx.d + 1), dtype=np.float32)
    _check(load().gempe_accumulators(ctx.handle, _ptr(out), out.size))
    return out[:, : ctx.d].copy(), out[:, ctx.d].copy()


def gempe_histograms(ctx: _Ctx, bins: int):
    out = np.empty(2 * bins, dtype=np.float32)
    _check(load().gempe_histograms(ctx.handle, _ptr(out), out.size))
    return out[:bins].copy(), out[bins:].copy()


def gempe_sample(ctx: _Ctx, loss_stream: bool = False, stream_id: int | None = None) -> np.ndarray:
    """stream_id: 0 the epoch's samples, 1 the loss estimator's, 2 the separate histogram pass's."""
    sid = (1 if loss_stream else 0) if stream_id is None else int(stream_id)
    out = np.empty(ctx.n * ctx.k, dtype=np.int32)
    _check(load().gempe_sample(ctx.handle, sid, _ptr(out), out.size))
    return out.reshape(ctx.n, ctx.k)


def gempe_is_edge(ctx: _Ctx, pairs) -> np.ndarray:
    pairs = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
    out = np.empty(len(pairs), dtype=np.uint8)
    _check(load().gempe_is_edge(ctx.handle, _ptr(pairs), len(pairs), _ptr(out)))
    return out.astype(bool)


def gempe_loss(ctx: _Ctx):
    pe = ctypes.c_double()
    s = ctypes.c_float()
    _check(load().gempe_loss(ctx.handle, ctypes.byref(pe), ctypes.byref(s)))
    return pe.value, s.value


def gempe_loss_exact(ctx: _Ctx, fit_sigma: bool = False):
    """Exact Eq. 2 over all pairs; with fit_sigma the minimum over sigma: (PE bits, sigma)."""
    pe = ctypes.c_double()
    s = ctypes.c_float()
    _check(load().gempe_loss_exact(ctx.handle, 1 if fit_sigma else 0, ctypes.byref(pe), ctypes.byref(s)))
    return pe.value, s.value


def gempe_fit_sigma(hist_e, hist_n, hist_max: float = 12.0, mu: float = 1.5, stream=None) -> float:
    h = np.ascontiguousarray(np.concatenate([hist_e, hist_n]), dtype=np.float32)
    out = ctypes.c_float()
    _check(load().gempe_fit_sigma(_ptr(h), len(h) // 2, float(hist_max), float(mu),
                                  _stream_handle(stream), ctypes.byref(out)))
    return out.value


def gempe_fit_sigma_static(hist_e, hist_n, hist_max: float = 12.0, mu: float = 1.5, stream=None) -> float:
    """gempe_fit_sigma without device allocation (static 4096-bin scratch)."""
    h = np.ascontiguousarray(np.concatenate([hist_e, hist_n]), dtype=np.float32)
    out = ctypes.c_float()
    _check(load().gempe_fit_sigma_static(_ptr(h), len(h) // 2, float(hist_max), float(mu),
                                         _stream_handle(stream), ctypes.byref(out)))
    return out.value


def gempe_kernel_times(ctx: _Ctx, enable: bool = True) -> tuple[float, float, float]:
    """Switch per-kernel event timing of gempe_sweep / gempe_update on or off;
    returns the last recorded epoch's (sweep, tiles, update) windows in ms."""
    out = (ctypes.c_float * 3)()
    _check(load().gempe_kernel_times(ctx.handle, 1 if enable else 0, out))
    return float(out[0]), float(out[1]), float(out[2])


def gempe_test_tile_wait(poll_limit: int) -> tuple[int, int]:
    """Test hook: one tile-shaped CTA whose bounded mbarrier wait runs out;
    (status it recorded, 1 if it freed its TMEM)."""
    st, fr = ctypes.c_int32(), ctypes.c_int32()
    _check(load().gempe_test_tile_wait(int(poll_limit), ctypes.byref(st), ctypes.byref(fr)))
    return st.value, fr.value


def gempe_stats(ctx: _Ctx) -> dict:
    s = gempe_stats_t()
    _check(load().gempe_stats(ctx.handle, ctypes.byref(s)))
    return {f: getattr(s, f) for f, _ in gempe_stats_t._fields_}


class _Batch:
    """Owned batch handle (gempe_batch_destroy on close / GC)."""

    def __init__(self, handle, ns, ds, keep=()):
        self.handle = handle
        self.ns, self.ds = list(ns), list(ds)
        self._keep = keep   # host CSR arrays and params stay alive with the handle

    def close(self):
        if self.handle:
            load().gempe_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def gempe_batch_create(graphs, params: gempe_params | None = None, stream=None) -> _Batch:
    """graphs: sequence of (row_ptr, col_idx, d)."""
    keep = []
    descs = (gempe_graph_desc * len(graphs))()
    ns, ds = [], []
    for q, (rp, ci, d) in enumerate(graphs):
        rp = np.ascontiguousarray(rp, dtype=np.int32)
        ci = np.ascontiguousarray(ci, dtype=np.int32)
        keep += [rp, ci]
        descs[q].row_ptr = rp.ctypes.data
        descs[q].col_idx = ci.ctypes.data if len(ci) else None
        descs[q].n = len(rp) - 1
        descs[q].d = int(d)
        ns.append(len(rp) - 1)
        ds.append(int(d))
    p = params or gempe_default_params()
    h = ctypes.c_void_p()
    _check(load().gempe_batch_create(len(graphs), descs, ctypes.byref(p), _stream_handle(stream), ctypes.byref(h)))
    return _Batch(h, ns, ds, keep=(p,))


def gempe_batch_destroy(b: _Batch) -> None:
    b.close()


def gempe_batch_step(b: _Batch, iters: int = 1) -> None:
    _check(load().gempe_batch_step(b.handle, int(iters)))


def gempe_batch_positions(b: _Batch, graph: int, out: np.ndarray | None = None) -> np.ndarray:
    """Positions of one graph of the batch; out: a float32 (n, d) array to fill
    (e.g. pinned host memory), else a new one."""
    if out is None:
        out = np.empty((b.ns[graph], b.ds[graph]), dtype=np.float32)
    if out.dtype != np.float32 or not out.flags.c_contiguous or out.size != b.ns[graph] * b.ds[graph]:
        raise ValueError("out must be a C-contiguous float32 array of n*d elements")
    _check(load().gempe_batch_positions(b.handle, int(graph), _ptr(out), out.size))
    return out


def gempe_batch_loss(b: _Batch, graph: int):
    pe = ctypes.c_double()
    s = ctypes.c_float()
    _check(load().gempe_batch_loss(b.handle, int(graph), ctypes.byref(pe), ctypes.byref(s)))
    return pe.value, s.value


def gempe_batch_stats(b: _Batch, graph: int) -> dict:
    s = gempe_stats_t()
    _check(load().gempe_batch_stats(b.handle, int(graph), ctypes.byref(s)))
    return {f: getattr(s, f) for f, _ in gempe_stats_t._fields_}


def gempe_batch_shape(b: _Batch, d: int) -> dict:
    out = (ctypes.c_int64 * 7)()
    _check(load().gempe_batch_shape(b.handle, int(d), out))
    return {"unit": out[0], "lanes": out[1], "blocks_per_sm": out[2], "grid": out[3], "graphs": out[4],
            "tuned_sweep_ns": out[5], "kernel": out[6]}


def gempe_job_bytes(n: int, nnz: int, d: int, params: gempe_params | None = None) -> int:
    p = params or gempe_default_params()
    return int(load().gempe_job_bytes(int(n), int(nnz), int(d), ctypes.byref(p)))


class _Server:
    """Owned server handle (gempe_server_destroy on close / GC)."""

    def __init__(self, handle, keep=()):
        self.handle = handle
        self.shapes = {}     # job id -> (n, d)
        self._keep = keep

    def close(self):
        if self.handle:
            load().gempe_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def gempe_server_create(hbm_budget_bytes: int, max_jobs: int = 32, params: gempe_params | None = None) -> _Server:
    p = params or gempe_default_params()
    h = ctypes.c_void_p()
    _check(load().gempe_server_create(int(hbm_budget_bytes), int(max_jobs), ctypes.byref(p), ctypes.byref(h)))
    return _Server(h, keep=(p,))


def gempe_server_destroy(s: _Server) -> None:
    s.close()


def gempe_server_submit(s: _Server, row_ptr, col_idx, d: int, epochs: int, seed: int) -> int:
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    desc = gempe_job_desc()
    desc.row_ptr = rp.ctypes.data
    desc.col_idx = ci.ctypes.data if len(ci) else None
    desc.n = len(rp) - 1
    desc.d = int(d)
    desc.epochs = int(epochs)
    desc.seed = int(seed)
    jid = ctypes.c_uint64()
    _check(load().gempe_server_submit(s.handle, ctypes.byref(desc), ctypes.byref(jid)))
    s.shapes[jid.value] = (len(rp) - 1, int(d))
    return jid.value


def _info(i: gempe_job_info) -> dict:
    return {f: getattr(i, f) for f, _ in gempe_job_info._fields_}


def gempe_server_poll(s: _Server, job_id: int) -> dict:
    info = gempe_job_info()
    _check(load().gempe_server_poll(s.handle, ctypes.c_uint64(job_id), ctypes.byref(info)))
    return _info(info)


def gempe_server_wait(s: _Server, job_id: int, timeout_ms: int = 60000) -> dict:
    info = gempe_job_info()
    _check(load().gempe_server_wait(s.handle, ctypes.c_uint64(job_id), int(timeout_ms), ctypes.byref(info)))
    return _info(info)


def gempe_server_result(s: _Server, job_id: int) -> np.ndarray:
    n, d = s.shapes.pop(job_id)
    out = np.empty((n, d), dtype=np.float32)
    _check(load().gempe_server_result(s.handle, ctypes.c_uint64(job_id), _ptr(out), out.size))
    return out


def gempe_server_stats(s: _Server) -> dict:
    out = (ctypes.c_int64 * 6)()
    _check(load().gempe_server_stats(s.handle, out))
    return {"queued": out[0], "running": out[1], "completed": out[2], "failed": out[3], "bytes_in_use": out[4],
            "peak_bytes_in_use": out[5]}


def gempe_set_shape(ctx: _Ctx, unit_pairs: int = 128, edge_chunk: int = 32, lanes: int = 0, blocks_per_sm: int = 0,
                    kernel: int = 0) -> None:
    arr = (ctypes.c_int32 * 5)(unit_pairs, edge_chunk, lanes, blocks_per_sm, kernel)
    _check(load().gempe_set_shape(ctx.handle, arr))


def gempe_get_shape(ctx: _Ctx) -> dict:
    out = (ctypes.c_int32 * 6)()
    _check(load().gempe_get_shape(ctx.handle, out))
    return {"unit_pairs": out[0], "edge_chunk": out[1], "lanes": out[2], "blocks_per_sm": out[3], "kernel": out[4],
            "grid": out[5]}


def gempe_last_error() -> str:
    return load().gempe_last_error().decode()


def torch_allocator(device=None):
    """(alloc, free) callbacks routing engine allocations through torch's caching allocator."""
    import torch
    dev = torch.cuda.current_device() if device is None else device

    @ALLOC_FN
    def _alloc(nbytes, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev)
        except Exception:
            return None

    @FREE_FN
    def _free(ptr, user):
        torch.cuda.caching_allocator_delete(ptr)

    return _alloc, _free
