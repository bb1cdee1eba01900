"""GEMPE CPU oracle (FP64) -- test infrastructure only.

Thin numpy wrappers around ``gempe_oracle.c``.  Only ``tests/``, the package
smoke check and the benchmark's CPU-baseline leg may import this module; the
CUDA engine and its Python binding never do.  See ``gempe_oracle.c`` for the
paper passages each function follows and for the readings taken where the
paper is silent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "gempe_oracle.c")
LIB = os.path.join(HERE, "libgempe_oracle.so")
LIB_OMP = os.path.join(HERE, "libgempe_oracle_omp.so")

_lib = None
_lib_omp = None

_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_f32p = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_c = ctypes


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, -O2, no fast-math)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(SRC) > os.path.getmtime(LIB):
        tmp = LIB + ".tmp%d" % os.getpid()
        res = subprocess.run(["gcc", "-O2", "-std=c11", "-fno-fast-math", "-ffp-contract=off",
                              "-shared", "-fPIC", "-o", tmp, SRC, "-lm"],
                             capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + res.stderr)
        os.replace(tmp, LIB)
    return LIB


def build_omp(force: bool = False) -> str:
    """The same source with OpenMP (-fopenmp): orc_epoch's vertex and tile
    loops over all host threads, shared sums by atomic additions.  Only the
    benchmark's CPU baseline runs it; the parity tests use the serial build."""
    if force or not os.path.exists(LIB_OMP) or os.path.getmtime(SRC) > os.path.getmtime(LIB_OMP):
        tmp = LIB_OMP + ".tmp%d" % os.getpid()
        res = subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-fno-fast-math", "-ffp-contract=off",
                              "-shared", "-fPIC", "-o", tmp, SRC, "-lm"],
                             capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError("oracle OpenMP build failed:\n" + res.stderr)
        os.replace(tmp, LIB_OMP)
    return LIB_OMP


def _load_omp():
    global _lib_omp
    if _lib_omp is not None:
        return _lib_omp
    lib = ctypes.CDLL(build_omp())
    _bind(lib)
    _lib_omp = lib
    return lib


def threads(parallel: bool = False) -> int:
    """Host threads orc_epoch runs on in the serial (1) or the OpenMP build."""
    return int((_load_omp() if parallel else _load()).orc_threads())


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    _bind(lib)
    _lib = lib
    return lib


def _bind(lib):
    I32, I64, U64, F64, F32 = _c.c_int32, _c.c_int64, _c.c_uint64, _c.c_double, _c.c_float
    sig = {
        "orc_philox4x32_10": (None, [_u32p, _u32p, _u32p]),
        "orc_init_positions": (None, [I32, I32, U64, F32, _f32p]),
        "orc_is_edge": (_c.c_int, [_i32p, _i32p, I32, I32]),
        "orc_h_basic": (F64, [F64, F64]),
        "orc_dl": (F64, [F64, F64, F64, _c.c_int]),
        "orc_parabola": (None, [F64, F64, F64, _c.c_int, _c.c_int, _c.c_int,
                                _c.POINTER(F64), _c.POINTER(F64)]),
        "orc_sample": (None, [_i32p, _i32p, I32, I32, U64, I32, I32, I32, _i32p]),
        "orc_epoch": (_c.c_int, [I32, _i32p, _i32p, I32, _f64p, F64, F64, I32, U64, I32, I32,
                                 I32, I32, I32, F64, I32, F64, _f64p, _f64p, _f64p, _f64p,
                                 _f64p, _i32p, _i64p, _f64p, I32, I32, _i32p, I32, I32, I32, I32, I32]),
        "orc_epoch_range": (_c.c_int, [I32, _i32p, _i32p, I32, _f64p, F64, F64, I32, U64, I32, I32,
                                       I32, I32, I32, F64, I32, F64, _f64p, _f64p, _f64p, _f64p,
                                       _f64p, _i32p, _i64p, _f64p, I32, I32, _i32p, I32, I32, I32, I32, I32,
                                       I32, I32]),
        "orc_bytemap_addr": (None, [I32, U64, I32, I32, _i32p, I64, _c.POINTER(_c.c_uint32),
                                    _c.POINTER(_c.c_uint32)]),
        "orc_block_partners": (None, [I32, I32, I32, U64, I32, _i32p]),
        "orc_edge_terms_edgelist": (None, [I32, _i32p, _i32p, I32, _f64p, F64, F64, I32, I32,
                                           _f64p, _f64p]),
        "orc_edge_terms_csr": (None, [I32, _i32p, _i32p, I32, _f64p, F64, F64, I32, I32,
                                      _f64p, _f64p]),
        "orc_surrogate_L": (F64, [I32, _i32p, _i32p, I32, _f64p, F64, F64, I32, _i32p]),
        "orc_dpe_dsigma": (F64, [_f64p, _f64p, I32, F64, F64, F64]),
        "orc_hist_pe": (F64, [_f64p, _f64p, I32, F64, F64, F64]),
        "orc_sigma_fit": (F64, [_f64p, _f64p, I32, F64, F64, F64, F64, I32]),
        "orc_loss_exact": (F64, [I32, _i32p, _i32p, I32, _f64p, F64, F64]),
        "orc_dpe_dsigma_exact": (F64, [I32, _i32p, _i32p, I32, _f64p, F64, F64]),
        "orc_sigma_fit_exact": (F64, [I32, _i32p, _i32p, I32, _f64p, F64, F64, F64, I32]),
        "orc_loss_sampled": (F64, [I32, _i32p, _i32p, I32, _f64p, F64, F64, I32, U64, I32, I32]),
        "orc_run": (_c.c_int, [I32, _i32p, _i32p, I32, _f64p, _c.POINTER(F64), F64, I32, I32,
                               U64, I32, I32, I32, I32, I32, F64, I32, F64, I32, _i64p, I32, I32, I32, I32,
                               I32, I32, I32, I32]),
        "orc_hist_pass": (_c.c_int, [I32, _i32p, _i32p, I32, _f64p, I32, U64, I32, I32, I32, F64, _f64p, _f64p]),
        "orc_vertex_terms": (_c.c_int, [I32, _i32p, _i32p, I32, _f64p, F64, F64, I32, U64, I32, I32, I32, I32,
                                        I32, I32, I32, I32, I32, _i32p, _f64p, _f64p, _f64p]),
    }
    sig["orc_threads"] = (_c.c_int, [])
    sig["orc_lcg_next"] = (_c.c_uint32, [_c.c_uint32])
    sig["orc_lcg_vertex"] = (I32, [_c.c_uint32, I32])
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args


# ---------------------------------------------------------------------------
# Defaults: mu = 1.5 (Sec. III.F), sigma0 = 1 (Fig. 4), and the readings.
# ---------------------------------------------------------------------------
MU = 1.5
SIGMA0 = 1.0
MAX_RETRIES = 32
Z_MIN = 1e-30
HIST_BINS = 1024
HIST_MAX = 12.0
INIT_RANGE = 1.0


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def philox4x32_10(ctr, key):
    out = np.zeros(4, dtype=np.uint32)
    _load().orc_philox4x32_10(np.ascontiguousarray(ctr, dtype=np.uint32),
                              np.ascontiguousarray(key, dtype=np.uint32), out)
    return out


def lcg_next(state):
    """Sec. III.C's LCG: the state after `state`."""
    return int(_load().orc_lcg_next(int(state) & 0xFFFFFFFF))


def lcg_vertex(state, n):
    """Fig. 2's vertex of an LCG state (FP32 float trick, n read as 0)."""
    return int(_load().orc_lcg_vertex(int(state) & 0xFFFFFFFF, int(n)))


def init_positions(n, d, seed, init_range=INIT_RANGE):
    x = np.zeros(n * d, dtype=np.float32)
    _load().orc_init_positions(n, d, seed, init_range, x)
    return x.reshape(n, d)


def is_edge(row_ptr, col_idx, i, j):
    return bool(_load().orc_is_edge(_i32(row_ptr), _i32(col_idx), int(i), int(j)))


def h_basic(n, m):
    return _load().orc_h_basic(float(n), float(m))


def dl(delta, mu, sigma, is_edge):
    return _load().orc_dl(float(delta), float(mu), float(sigma), int(bool(is_edge)))


def parabola(delta, mu, sigma, is_edge, w_formula=0, clamp_neg_d=1):
    d = ctypes.c_double()
    w = ctypes.c_double()
    _load().orc_parabola(float(delta), float(mu), float(sigma), int(bool(is_edge)), int(w_formula),
                         int(clamp_neg_d), ctypes.byref(d), ctypes.byref(w))
    return d.value, w.value


def sample(row_ptr, col_idx, epoch, seed, k, max_retries=MAX_RETRIES, loss_stream=False):
    n = len(row_ptr) - 1
    out = np.zeros(n * max(k, 1), dtype=np.int32)
    _load().orc_sample(_i32(row_ptr), _i32(col_idx), n, epoch, seed, int(loss_stream), k,
                       max_retries, out)
    return out[: n * k].reshape(n, k)


def block_partners(n, tile, epoch_idx, seed, P):
    out = np.zeros(P, dtype=np.int32)
    _load().orc_block_partners(n, tile, epoch_idx, seed, P, out)
    return out


def epoch(row_ptr, col_idx, x, sigma, epoch_idx, seed, k, mu=MU, max_retries=MAX_RETRIES,
          symmetric=1, w_formula=0, clamp_neg_d=1, z_min=Z_MIN, hist_bins=HIST_BINS,
          hist_max=HIST_MAX, block_partners=0, tile_vertices=128, per_slot=0, membership=0, bytemap_log2=24,
          rename_every=0, rng=0, anchors=None):
    """One epoch of Fig. 4; returns a dict of FP64 results.  ``abs_terms[i]`` is the
    sum of the sizes of the pair terms of y_i - z_i x_i (the scale of that sum's
    rounding when its terms cancel).  per_slot=1: Sec. III.C's policy, one
    sample per CSR slot (``samples`` then has one entry per slot).  rng=1: Sec. III.C's
    LCG draws the sampled non-edges (seeded per slot from Philox).  anchors=(lo, hi):
    the terms of those anchors alone (y, z, histograms and counts of their pairs;
    x_new is then not an epoch's)."""
    n = len(row_ptr) - 1
    nnz = int(row_ptr[-1])
    x = _f64(x)
    d = x.shape[1]
    y = np.zeros((n, d)); z = np.zeros(n); xn = np.zeros((n, d))
    he = np.zeros(hist_bins); hn = np.zeros(hist_bins)
    smp = np.zeros(max(nnz, 1) if per_slot else n * max(k, 1), dtype=np.int32)
    st = np.zeros(5, dtype=np.int64)
    absd = np.zeros(n)
    n_tiles = (n + tile_vertices - 1) // tile_vertices
    parts = np.zeros(max(1, n_tiles * block_partners), dtype=np.int32)
    args = (n, _i32(row_ptr), _i32(col_idx), d, x, sigma, mu, epoch_idx, seed, k,
            max_retries, symmetric, w_formula, clamp_neg_d, z_min, hist_bins,
            hist_max, y, z, xn, he, hn, smp, st, absd, block_partners,
            tile_vertices, parts, per_slot, membership, bytemap_log2, rename_every, rng)
    if anchors is None:
        rc = _load().orc_epoch(*args)
    else:
        rc = _load().orc_epoch_range(*args, int(anchors[0]), int(anchors[1]))
    if rc == -2:
        raise ValueError("anchor range outside [0, n)")
    if rc != 0:
        raise MemoryError("oracle epoch failed")
    samples = smp[:nnz] if per_slot else smp[: n * k].reshape(n, k)
    return dict(y=y, z=z, x_new=xn, hist_e=he, hist_n=hn, samples=samples,
                accepted=int(st[0]), rejected=int(st[1]), exhausted=int(st[2]), draws=int(st[3]),
                false_pos=int(st[4]),
                delta=y - z[:, None] * x, abs_terms=absd,
                partners=parts[: n_tiles * block_partners].reshape(n_tiles, block_partners)
                if block_partners else None)


def vertex_terms(row_ptr, col_idx, x, sigma, epoch_idx, seed, k, query, mu=MU, max_retries=MAX_RETRIES,
                 symmetric=1, w_formula=0, clamp_neg_d=1, z_min=Z_MIN, block_partners=0, tile_vertices=128,
                 per_slot=0):
    """Eq. 3 for the vertices ``query`` alone (distinct ids), with the samples
    ``epoch`` draws: rows of y, z, delta = y - z x, abs_terms and x_new in the
    order of ``query``.  For checks at sizes where a whole epoch here is slow."""
    n = len(row_ptr) - 1
    x = _f64(x)
    d = x.shape[1]
    q = _i32(query)
    y = np.zeros((len(q), d)); z = np.zeros(len(q)); absd = np.zeros(len(q))
    rc = _load().orc_vertex_terms(n, _i32(row_ptr), _i32(col_idx), d, x, sigma, mu, epoch_idx, seed, k,
                                  max_retries, symmetric, w_formula, clamp_neg_d, block_partners, tile_vertices,
                                  per_slot, len(q), q, y, z, absd)
    if rc == -2:
        raise ValueError("query ids must be distinct vertices")
    if rc != 0:
        raise MemoryError("oracle vertex terms failed")
    xq = x[q]
    x_new = np.where((z >= z_min)[:, None], y / np.maximum(z, 1e-300)[:, None], xq)
    return dict(y=y, z=z, delta=y - z[:, None] * xq, abs_terms=absd, x_new=x_new)


def edge_terms(row_ptr, col_idx, x, sigma, mu=MU, w_formula=0, clamp_neg_d=1, form="csr"):
    n = len(row_ptr) - 1
    x = _f64(x)
    d = x.shape[1]
    y = np.zeros((n, d)); z = np.zeros(n)
    f = _load().orc_edge_terms_csr if form == "csr" else _load().orc_edge_terms_edgelist
    f(n, _i32(row_ptr), _i32(col_idx), d, x, sigma, mu, w_formula, clamp_neg_d, y, z)
    return y, z


def surrogate_L(row_ptr, col_idx, x, sigma, samples, mu=MU):
    n = len(row_ptr) - 1
    x = _f64(x)
    samples = _i32(samples)
    k = samples.shape[1] if samples.ndim == 2 else 0
    return _load().orc_surrogate_L(n, _i32(row_ptr), _i32(col_idx), x.shape[1], x, sigma, mu, k,
                                   samples.reshape(-1) if k else np.zeros(1, np.int32))


def dpe_dsigma(hist_e, hist_n, hist_max, mu, sigma):
    he, hn = _f64(hist_e), _f64(hist_n)
    return _load().orc_dpe_dsigma(he, hn, len(he), hist_max, mu, sigma)


def hist_pe(hist_e, hist_n, hist_max, mu, sigma):
    he, hn = _f64(hist_e), _f64(hist_n)
    return _load().orc_hist_pe(he, hn, len(he), hist_max, mu, sigma)


def sigma_fit(hist_e, hist_n, hist_max=HIST_MAX, mu=MU, lo=1e-3, hi=1e3, iters=60):
    he, hn = _f64(hist_e), _f64(hist_n)
    return _load().orc_sigma_fit(he, hn, len(he), hist_max, mu, lo, hi, iters)


def loss_exact(row_ptr, col_idx, x, sigma, mu=MU):
    x = _f64(x)
    return _load().orc_loss_exact(len(row_ptr) - 1, _i32(row_ptr), _i32(col_idx), x.shape[1], x,
                                  sigma, mu)


def dpe_dsigma_exact(row_ptr, col_idx, x, sigma, mu=MU):
    """dPE/dsigma over all pairs, times N (the number of unordered pairs)."""
    x = _f64(x)
    return _load().orc_dpe_dsigma_exact(len(row_ptr) - 1, _i32(row_ptr), _i32(col_idx), x.shape[1], x, mu, sigma)


def sigma_fit_exact(row_ptr, col_idx, x, mu=MU, lo=1e-3, hi=1e3, iters=60):
    """The slope minimising the exact Eq. 2 (bisection on the exact derivative)."""
    x = _f64(x)
    return _load().orc_sigma_fit_exact(len(row_ptr) - 1, _i32(row_ptr), _i32(col_idx), x.shape[1], x, mu,
                                       lo, hi, iters)


def bytemap_addr(n, seed, period, log2_size, pairs):
    """Byte-map addresses of (i, j) pairs under the renaming of `period`, and (a, b) of that renaming."""
    pairs = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
    out = np.zeros(len(pairs), dtype=np.uint32)
    ab = np.zeros(2, dtype=np.uint32)
    _load().orc_bytemap_addr(n, seed, period, log2_size, pairs.ravel(), len(pairs),
                             out.ctypes.data_as(_c.POINTER(_c.c_uint32)), ab.ctypes.data_as(_c.POINTER(_c.c_uint32)))
    return out, (int(ab[0]), int(ab[1]))


def hist_pass(row_ptr, col_idx, x, epoch_idx, seed, k, max_retries=MAX_RETRIES, hist_bins=HIST_BINS,
              hist_max=HIST_MAX):
    """Sec. III.F's separate histogram pass: all edges and k fresh samples per vertex at x."""
    x = _f64(x)
    he = np.zeros(hist_bins)
    hn = np.zeros(hist_bins)
    rc = _load().orc_hist_pass(len(row_ptr) - 1, _i32(row_ptr), _i32(col_idx), x.shape[1], x, epoch_idx, seed, k,
                               max_retries, hist_bins, hist_max, he, hn)
    if rc != 0:
        raise MemoryError("oracle histogram pass failed")
    return he, hn


def loss_sampled(row_ptr, col_idx, x, sigma, epoch_idx, seed, k, mu=MU, max_retries=MAX_RETRIES):
    x = _f64(x)
    return _load().orc_loss_sampled(len(row_ptr) - 1, _i32(row_ptr), _i32(col_idx), x.shape[1], x,
                                    sigma, mu, epoch_idx, seed, k, max_retries)


def run(row_ptr, col_idx, x, sigma, epochs, seed, k, epoch0=0, mu=MU, max_retries=MAX_RETRIES,
        symmetric=1, w_formula=0, clamp_neg_d=1, z_min=Z_MIN, hist_bins=HIST_BINS,
        hist_max=HIST_MAX, sigma_every=1, block_partners=0, tile_vertices=128, per_slot=0, sigma_source=0, membership=0,
        bytemap_log2=24, rename_every=0, parallel=False, rng=0):
    """Fig. 4 for ``epochs`` iterations from state (x, sigma); returns (x, sigma, stats).
    parallel: the OpenMP build (all host threads; sums in another order)."""
    n = len(row_ptr) - 1
    x = np.array(x, dtype=np.float64, order="C", copy=True)
    s = ctypes.c_double(sigma)
    st = np.zeros(5, dtype=np.int64)
    rc = (_load_omp() if parallel else _load()).orc_run(n, _i32(row_ptr), _i32(col_idx), x.shape[1], x, ctypes.byref(s), mu,
                         epoch0, epochs, seed, k, max_retries, symmetric, w_formula, clamp_neg_d,
                         z_min, hist_bins, hist_max, sigma_every, st, block_partners, tile_vertices, per_slot, sigma_source,
                         membership, bytemap_log2, rename_every, rng)
    if rc != 0:
        raise MemoryError("oracle run failed")
    return x, s.value, dict(accepted=int(st[0]), rejected=int(st[1]), exhausted=int(st[2]), false_pos=int(st[4]))
