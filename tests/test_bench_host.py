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
    assert rec == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3,
                   "samples_under_load": 3}


def test_clock_record_takes_the_median_under_load():
    """Samples with the GPU idle (utilisation 0, e.g. while the host builds a
    graph) do not pull the median clock down; reasons come from every sample."""
    rows = [r.split(", ") for r in (
        "0, 345, 2070, 100.0, 0x0, Not Active, Not Active, Not Active, Not Active, 0",
        "0, 345, 2070, 100.0, 0x0, Not Active, Not Active, Not Active, Not Active, 0",
        "0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active, 97",
        "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active, 100")]
    rec = bench.ClockSampler.parse(rows)
    assert rec["sm_mhz"] == 2025.0 and rec["samples"] == 4 and rec["samples_under_load"] == 2
    assert rec["reasons"] == ["sw_power_cap"]


def test_model_bytes_follow_the_per_unit_figures():
    """The roofline numerator: edges 2m (4 + R), samples S (R + (d+1) 4) and
    per vertex n (4 + R + (d+1) 4) for the sweep, 32 B per sample for the
    sampler, P (R + (d+1) 4) per tile, and the update's accumulator read and
    position writes.  R-MAT scale 16 (m = 910,301, S = 655,360, d = 2):
    36.5 MB for the sweep and 58.8 MB for the whole epoch."""
    mb = bench.model_bytes(65536, 910301, 2, 0, samples=655360)
    assert mb["sweep"] == 2 * 910301 * 12 + 655360 * 20 + 65536 * 24
    assert abs(mb["sweep"] / 1e6 - 36.5) < 0.05
    assert abs(mb["epoch"] / 1e6 - 58.8) < 0.05
    # the BA workload, FP32 and BF16 (R = 4d, 2d), block tiles of 64 partners
    n, m, d, t = 1000000, 7999964, 64, 7813
    f32 = bench.model_bytes(n, m, d, 0, tiles=t)
    b16 = bench.model_bytes(n, m, d, 1, tiles=t)
    assert f32["tiles"] == t * 64 * (256 + 260) and b16["tiles"] == t * 64 * (128 + 260)
    assert f32["sweep"] - b16["sweep"] == (2 * m + n) * 128
    assert b16["update"] - f32["update"] == n * 6 * d
    assert f32["sampler"] == 0 and f32["epoch"] == f32["sweep"] + f32["tiles"] + f32["update"]
    assert bench.tile_flops(t, d) == t * 128 * 64 * 7 * d


def test_job_shares_cover_every_job_once_and_balance():
    rng = __import__("numpy").random.default_rng(3)
    sizes = [int(v) for v in rng.integers(1, 1000, 257)]
    for world in (1, 2, 3, 4, 8):
        shares = [bench.shard_jobs(sizes, world, r) for r in range(world)]
        flat = sorted(q for s in shares for q in s)
        assert flat == list(range(len(sizes)))
        loads = [sum(sizes[q] for q in s) for s in shares]
        assert max(loads) - min(loads) <= max(sizes)
        streams = [bench.stream_share(101, world, r) for r in range(world)]
        assert sorted(q for s in streams for q in s) == list(range(101))


def test_openmp_oracle_matches_the_serial_oracle(oracle_mod, sbm_1000):
    """The timed CPU baseline (the oracle's source built with OpenMP) computes
    the same epoch as the parity oracle: the same samples and counts, sums
    equal up to the order of FP64 additions."""
    import numpy as np
    rp, ci = sbm_1000["row_ptr"], sbm_1000["col_idx"]
    for d, kw in ((2, dict(k=5)), (16, dict(k=0, block_partners=64))):
        x0 = oracle_mod.init_positions(1000, d, 9)
        k = kw.pop("k")
        a = oracle_mod.run(rp, ci, x0, 1.0, 1, 9, k, **kw)
        b = oracle_mod.run(rp, ci, x0, 1.0, 1, 9, k, parallel=True, **kw)
        assert a[2] == b[2]
        np.testing.assert_allclose(b[0], a[0], rtol=1e-10, atol=1e-12 * np.abs(a[0]).max())
        assert b[1] == __import__("pytest").approx(a[1], rel=1e-9)
    assert oracle_mod.threads(parallel=False) == 1 and oracle_mod.threads(parallel=True) >= 1
