"""The C ABI from a plain C99 program: include/gempe.h compiles as C, the
library links, and the calls that need no GPU behave as documented
(defaults of the paper, host CSR validation naming the failing pair,
checkpoint argument checks, thread-local error messages)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "gempe.h"

int main(void) {
    gempe_params p;
    gempe_default_params(&p);
    printf("defaults %.2f %.2f %d %d %d\n", p.mu, p.sigma0, p.sigma_every, p.neg_per_vertex, p.max_retries);
    /* a triangle 0-1-2 plus the edge 2-3 */
    const int32_t rp[5] = {0, 2, 4, 7, 8};
    const int32_t ci[8] = {1, 2, 0, 2, 0, 1, 3, 2};
    printf("valid %d\n", (int)gempe_validate_csr(rp, ci, 4));
    /* row 2 lists 3 but row 3 does not list 2 back */
    const int32_t ci_bad[8] = {1, 2, 0, 2, 0, 1, 3, 1};
    gempe_status st = gempe_validate_csr(rp, ci_bad, 4);
    printf("invalid %d [%s]\n", (int)st, gempe_last_error());
    size_t len = 0;
    printf("save-null %d\n", (int)gempe_save(NULL, NULL, &len));
    return 0;
}
"""


def test_header_compiles_as_c_and_links():
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    from paper_2011_03479_gb300 import binding
    lib = binding.load()   # builds libgempe.so when needed
    libdir = os.path.dirname(lib._name)
    cuda_lib = "/usr/local/cuda/lib64"
    import tempfile
    with tempfile.TemporaryDirectory() as tmp:
        src = os.path.join(tmp, "consumer.c")
        exe = os.path.join(tmp, "consumer")
        with open(src, "w") as f:
            f.write(PROGRAM)
        cmd = [gcc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), src, "-o", exe,
               "-L", libdir, "-lgempe", f"-Wl,-rpath,{libdir}"]
        if os.path.isdir(cuda_lib):
            cmd += ["-L", cuda_lib, f"-Wl,-rpath,{cuda_lib}"]
        res = subprocess.run(cmd, capture_output=True, text=True)
        assert res.returncode == 0, res.stderr
        out = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stderr
    lines = out.stdout.splitlines()
    assert lines[0] == "defaults 1.50 1.00 1 5 32"
    assert lines[1] == "valid 0"
    assert lines[2].startswith("invalid -2 [") and "symmetric" in lines[2] and "(2,3)" in lines[2]
    assert lines[3] == "save-null -1"
