"""In-tree build of the package's native libraries.

* ``inputs/libgraphgen.so``  - seeded synthetic graph generators (plain C, gcc)
* ``libgempe.so``            - the GEMPE epoch engine: sm_103a CUDA kernels plus
                               the C-ABI declared in ``include/gempe.h`` (nvcc)

Both are rebuilt only when a source is newer than the library.  nvcc
cross-compiles for sm_103a without a GPU; the CUDA translation units are
compiled in parallel and linked with ``nvcc -shared``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
GRAPHGEN_SRC = os.path.join(PKG, "inputs", "graphgen.c")
GRAPHGEN_LIB = os.path.join(PKG, "inputs", "libgraphgen.so")
GEMPE_LIB = os.path.join(PKG, "libgempe.so")
BUILD_DIR = os.path.join(PKG, "_build")

ARCH_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC",
              "-Xcompiler", "-fvisibility=hidden", "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the GEMPE CUDA engine cannot be built")


def _stale(target: str, sources: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in sources)


def _run(cmd: list[str]) -> None:
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("build failed: " + " ".join(cmd) + "\n" + res.stdout + res.stderr)


def build_graphgen(force: bool = False) -> str:
    if force or _stale(GRAPHGEN_LIB, [GRAPHGEN_SRC]):
        tmp = GRAPHGEN_LIB + ".tmp%d" % os.getpid()
        _run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, GRAPHGEN_SRC, "-lm"])
        os.replace(tmp, GRAPHGEN_LIB)
    return GRAPHGEN_LIB


def cuda_sources() -> list[str]:
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _headers() -> list[str]:
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    hs += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    return hs


def build_gempe(force: bool = False, verbose_ptxas: bool = False) -> str:
    srcs = cuda_sources()
    if not (force or _stale(GEMPE_LIB, srcs + _headers())):
        return GEMPE_LIB
    os.makedirs(BUILD_DIR, exist_ok=True)
    nvcc = _nvcc()
    extra = ["-Xptxas", "-v"] if verbose_ptxas else []

    def compile_one(src: str) -> str:
        obj = os.path.join(BUILD_DIR, os.path.basename(src) + ".o")
        _run([nvcc, *ARCH_FLAGS, *NVCC_FLAGS, *extra, "-I", INCLUDE, "-I", CSRC,
              "-c", src, "-o", obj])
        return obj

    with ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 1))) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = GEMPE_LIB + ".tmp%d" % os.getpid()
    _run([nvcc, *ARCH_FLAGS, "-shared", "-o", tmp, *objs, "-lcudart"])
    os.replace(tmp, GEMPE_LIB)
    return GEMPE_LIB


def build_all(force: bool = False) -> None:
    build_graphgen(force)
    build_gempe(force)
