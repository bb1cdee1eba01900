"""Host-side logic of bench.py that needs no GPU."""
import os
import shutil

import bench


def test_kernel_hash_ignores_the_abi_front_ends(tmp_path):
    """The profile summaries' DRAM traffic is keyed by a hash of the sources
    that define the kernels and their launch shapes: editing a C-ABI front
    end keeps it, editing a kernel or the launch configuration changes it."""
    src = os.path.join(bench.ROOT, "paper_2011_03479_gb300", "csrc")
    dst = tmp_path / "csrc"
    shutil.copytree(src, dst)
    h0 = bench.kernel_source_hash(str(dst))
    assert h0 == bench.kernel_source_hash()
    for fn in sorted(bench.ABI_FRONT_ENDS):
        with open(dst / fn, "a") as f:
            f.write("\n// edited\n")
    assert bench.kernel_source_hash(str(dst)) == h0
    for fn in ("kernels.cu", "pack.cu"):
        with open(dst / fn, "a") as f:
            f.write("\n// edited\n")
        h1 = bench.kernel_source_hash(str(dst))
        assert h1 != h0
        h0 = h1


def test_abi_front_ends_hold_no_device_code():
    src = os.path.join(bench.ROOT, "paper_2011_03479_gb300", "csrc")
    for fn in bench.ABI_FRONT_ENDS:
        text = open(os.path.join(src, fn)).read()
        assert "__global__" not in text and "__device__" not in text and "<<<" not in text, fn


def test_byte_model_uses_the_rows_the_form_reads():
    """The sweep's algorithmic bytes charge a position row at the size the
    form reads: BF16 (2d) for the precision form at d >= 8, FP32 (4d)
    otherwise; with no samples the two differ by exactly the own rows and
    one neighbour row per CSR slot."""
    assert bench.position_row_bytes(64, 1) == 128 and bench.position_row_bytes(64, 0) == 256
    assert bench.position_row_bytes(2, 1) == 8      # d <= 4 stays FP32
    n, nnz, d = 1000, 16000, 64
    b16 = bench.sweep_algorithmic_bytes(n, nnz, d, 0, 300, 0, row_bytes=bench.position_row_bytes(d, 1))
    b32 = bench.sweep_algorithmic_bytes(n, nnz, d, 0, 300, 0)
    assert b32 - b16 == (n + nnz) * 2 * d


def test_clock_sampler_reads_clocks_and_reasons(tmp_path, monkeypatch):
    """The clocks record beside every bench line: median SM clock under load,
    the maximum, and every throttle reason seen active, parsed from
    nvidia-smi's CSV (a stand-in script prints three samples here)."""
    import time
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/sh\n"
                    "echo '0, 1965, 2070, 900.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active'\n"
                    "echo '0, 2070, 2070, 950.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active'\n"
                    "echo '0, 2070, 2070, 960.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active'\n"
                    "exec sleep 30\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ.get('PATH', '')}")
    cs = bench.ClockSampler(0)
    cs.start()
    deadline = time.time() + 10
    while time.time() < deadline and sum(1 for _ in open(cs.path)) < 3:
        time.sleep(0.05)
    rec = cs.stop()
    assert rec == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
