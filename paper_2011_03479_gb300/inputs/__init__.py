"""Seeded synthetic graphs shaped like the paper's workloads.

The paper evaluates on the world flight network, the California road network,
BlogCatalog, Cora, PubMed and power-law graphs from a Java generator; none of
them is available here, so seeded synthetic graphs stand in for them:

* ``sbm``               stochastic block model (community graphs, drawing)
* ``rmat``              R-MAT power-law graph (graph drawing at scale)
* ``barabasi_albert``   preferential-attachment graph (representation learning)

Each returns ``(row_ptr, col_idx)`` as int32 numpy arrays: a symmetric CSR
matrix with sorted rows, no self loops and no duplicates.  This module holds
none of the embedding method's arithmetic.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .. import _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build_graphgen()
        lib = ctypes.CDLL(path)
        i32p = ctypes.POINTER(ctypes.c_int32)
        out = [ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(i32p), ctypes.POINTER(i32p),
               ctypes.POINTER(ctypes.c_int64)]
        lib.gg_sbm.argtypes = [ctypes.c_int32, i32p, ctypes.c_double, ctypes.c_double,
                               ctypes.c_uint64, *out]
        lib.gg_rmat.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, ctypes.c_uint64, *out]
        lib.gg_barabasi_albert.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, *out]
        for f in (lib.gg_sbm, lib.gg_rmat, lib.gg_barabasi_albert):
            f.restype = ctypes.c_int
        lib.gg_free.argtypes = [ctypes.c_void_p]
        lib.gg_free.restype = None
        _lib = lib
    return _lib


def _call(fn, *args):
    lib = _load()
    n = ctypes.c_int32(0)
    rp = ctypes.POINTER(ctypes.c_int32)()
    ci = ctypes.POINTER(ctypes.c_int32)()
    nnz = ctypes.c_int64(0)
    rc = fn(*args, ctypes.byref(n), ctypes.byref(rp), ctypes.byref(ci), ctypes.byref(nnz))
    if rc != 0:
        raise RuntimeError(f"graph generator failed with code {rc}")
    try:
        row_ptr = np.ctypeslib.as_array(rp, shape=(n.value + 1,)).copy()
        col_idx = (np.ctypeslib.as_array(ci, shape=(nnz.value,)).copy() if nnz.value
                   else np.zeros(0, dtype=np.int32))
    finally:
        lib.gg_free(ctypes.cast(rp, ctypes.c_void_p))
        lib.gg_free(ctypes.cast(ci, ctypes.c_void_p))
    return row_ptr, col_idx


def sbm(block_sizes, p_in: float, p_out: float, seed: int):
    sizes = np.ascontiguousarray(block_sizes, dtype=np.int32)
    return _call(_load().gg_sbm, len(sizes), sizes.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                 float(p_in), float(p_out), ctypes.c_uint64(seed))


def rmat(scale: int, edge_factor: int, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 1):
    return _call(_load().gg_rmat, int(scale), int(edge_factor), float(a), float(b), float(c),
                 ctypes.c_uint64(seed))


def barabasi_albert(n: int, m: int, seed: int):
    return _call(_load().gg_barabasi_albert, int(n), int(m), ctypes.c_uint64(seed))


# ---------------------------------------------------------------------------
# Named workloads (sizes of the paper's drawing / representation settings)
# ---------------------------------------------------------------------------
# Philox key of the embedding run for each workload (the graph seeds differ).
EMBED_SEED = 0x6E6D7065


def sbm_1000():
    """SBM, n=1,000 in 4 blocks of 250, p_in=0.05, p_out=0.002; d=2, k=5, 200 epochs."""
    rp, ci = sbm([250, 250, 250, 250], 0.05, 0.002, seed=1001)
    return dict(name="sbm-n1000-b4", row_ptr=rp, col_idx=ci, d=2, k=5, epochs=200)


def rmat_s16():
    """R-MAT scale 16, edge factor 16, (a,b,c,d)=(.57,.19,.19,.05); d=2, k=10, 500 epochs."""
    rp, ci = rmat(16, 16, 0.57, 0.19, 0.19, seed=2001)
    return dict(name="rmat-s16-ef16", row_ptr=rp, col_idx=ci, d=2, k=10, epochs=500)


def ba_1m():
    """Barabasi-Albert n=1,000,000, m=8; d=64, 100 epochs."""
    rp, ci = barabasi_albert(1_000_000, 8, seed=3001)
    return dict(name="ba-n1m-m8", row_ptr=rp, col_idx=ci, d=64, k=10, epochs=100)


def ba_300k():
    """Barabasi-Albert n=300,000, m=8 (the BA workload's kernels at a size for full profiler captures)."""
    rp, ci = barabasi_albert(300_000, 8, seed=3001)
    return dict(name="ba-n300k-m8", row_ptr=rp, col_idx=ci, d=64, k=10, epochs=100)


def sbm_batch(count: int, n_lo: int, n_hi: int, dims=(2, 16, 64), deg_lo: float = 4.0, deg_hi: float = 32.0,
              blocks_lo: int = 2, blocks_hi: int = 8, intra: float = 0.9, seed: int = 4000):
    """`count` independent SBM graphs: n log-uniform in [n_lo, n_hi], blocks
    uniform in [blocks_lo, blocks_hi] (equal sizes, remainder spread), mean
    degree uniform in [deg_lo, deg_hi] with a fraction `intra` of it inside
    the vertex's block, d drawn from `dims`.  Graph q uses generator seed
    seed + 1 + q; the shape parameters come from a numpy Generator(seed)."""
    rng = np.random.default_rng(seed)
    out = []
    for q in range(count):
        n = int(round(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi)))))
        nb = int(rng.integers(blocks_lo, blocks_hi + 1))
        nb = max(1, min(nb, n // 2))
        deg = float(rng.uniform(deg_lo, deg_hi))
        d = int(rng.choice(np.asarray(dims)))
        sizes = np.full(nb, n // nb, dtype=np.int64)
        sizes[: n % nb] += 1
        bs = n / nb
        p_in = min(1.0, intra * deg / max(bs - 1.0, 1.0))
        p_out = min(1.0, (1.0 - intra) * deg / max(n - bs, 1.0)) if nb > 1 else 0.0
        rp, ci = sbm(sizes, p_in, p_out, seed=seed + 1 + q)
        out.append(dict(row_ptr=rp, col_idx=ci, d=d, n=n, blocks=nb, mean_degree=deg))
    return out


def sbm_batch_256():
    """256 SBMs, n log-uniform in [500, 50,000], 2-8 blocks, mean degree
    U[4, 32] (90% inside the block), d in {2, 16, 64}; k=5, 200 epochs."""
    return dict(name="sbm-batch-256", graphs=sbm_batch(256, 500, 50_000), k=5, epochs=200)


WORKLOADS = {"sbm-n1000-b4": sbm_1000, "rmat-s16-ef16": rmat_s16, "ba-n1m-m8": ba_1m, "ba-n300k-m8": ba_300k}
