#!/usr/bin/env python3
"""GEMPE epoch benchmark: pair-updates per second of one GEMPE epoch, plain
FP32 against the BF16 / batched / served forms, and the per-graph embed
latency of serving.

Headline (default): the representation-learning workload ba-n1m-m8 -- a
Barabasi-Albert graph with n = 1,000,000 and m = 8 (about 8.0 M edges),
d = 64, block-sampled non-edges (tiles of 128 vertices x 64 partners), 100
epochs per job.  `value` is the plain FP32 run (FP32 positions and
arithmetic, the paper's precision); beside it the BF16 form of the same seed
(BF16 positions on tensor-core tiles, FP32 master positions and sums) with
its own timing and the ratio between the two.  Nested records in the same
line: the graph-drawing workload (R-MAT scale 16, d = 2), the batched form
(256 SBM graphs, one CUDA-graph launch per epoch) and the served form
(Poisson arrivals, p50/p99 latency).  Synthetic, seeded inputs.

A step is one epoch (pair sweep + tiles + position update + sigma refit)
through the C ABI (gempe_step(ctx, 1): one replay of the captured epoch
graph) on a torch CUDA stream, timed with CUDA events on that stream; the L2
cache is flushed (a 256 MiB write) between steps, outside the events.  A
second pass of as many epochs, as gempe_sweep + gempe_update with the
library's per-kernel events (gempe_kernel_times), gives each kernel's window
for the roofline.  Pair-updates per epoch = m undirected edges + the
sampled non-edges the epoch consumed.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gempe|reference]
                    [--workload NAME] [--no-nested]

--impl reference times the FP64 CPU oracle (the method restated in plain C,
OpenMP build over all host threads) on a bounded sample of the headline
workload.  Under torchrun (N > 1) every rank runs the single-graph workloads
as independent replicas (no collective on the data path) and takes its share
of the batch's graphs and of the served job stream; value is the sum of all
ranks' pair-updates over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pair-updates/sec per GEMPE epoch vs plain FP32 GPU; p50/p99 per-graph embed latency"
UNIT = "pair-updates/s"
HEADLINE = "ba-n1m-m8"
# engine parameters of each workload (the graph and d, k come from inputs.WORKLOADS)
FORMS = {
    "rmat-s16-ef16": {},
    "ba-n1m-m8": {"block_partners": 64, "precision": 1},          # BF16 + tensor-core tiles
    "ba-n1m-m8-fp32": {"block_partners": 64, "precision": 0},     # the plain FP32 run of the same seed (FP32 tiles)
    "ba-n300k-m8": {"block_partners": 64, "precision": 1},        # the same kernels at a size for full ncu captures
    "ba-n300k-m8-fp32": {"block_partners": 64, "precision": 0},
    # batched form: 256 SBM graphs, d in {2, 16, 64}, one CUDA-graph launch per epoch
    "sbm-batch-256": {"autotune": 1},
    "sbm-batch-256-bf16": {"autotune": 1, "precision": 1},         # BF16 positions for the d >= 8 graphs
}
BATCH_WORKLOADS = {"sbm-batch-256", "sbm-batch-256-bf16"}
# serving form: Poisson arrivals (50 jobs/s) of R-MAT embedding jobs under a 120 GB device budget
SERVE_WORKLOADS = {"rmat-serve-poisson50": {},
                   "rmat-serve-poisson50-bf16": {"precision": 1}}   # BF16 positions for the d >= 8 jobs
SERVE_MAX_JOBS = 600   # jobs of one serving run (12 s of arrivals at 50 per second)
FORMS.update(SERVE_WORKLOADS)
L2_FLUSH_BYTES = 256 << 20
UNIT_PAIRS = 128     # edge + sample slots per packed work unit of the d <= 4 sweep
BLOCK_P, BLOCK_T = 64, 128
# FP32 CUDA-core peak: 152 SMs x 128 FP32 lanes x 2 flops (FMA) x 2.07 GHz
SM_COUNT, FP32_LANES_PER_SM, SM_MAX_GHZ = 152, 128, 2.07
FP32_PEAK_TFLOPS = SM_COUNT * FP32_LANES_PER_SM * 2 * SM_MAX_GHZ / 1e3


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# Byte and flop models (no-reuse model: every random row gather paid once at
# its minimum size; own rows, CSR and accumulators streamed once).
# ---------------------------------------------------------------------------
def position_row_bytes(d, precision):
    """Bytes of the position row the pair arithmetic reads: the BF16 shadow
    (2d) in the precision form (d >= 8), else the FP32 positions (4d)."""
    return 2 * d if precision and d >= 8 else 4 * d


def model_bytes(n, m, d, precision=0, samples=0, tiles=0, partners=BLOCK_P):
    """Algorithmic bytes of one epoch per kernel, R the position row:
      sweep    edges 2m (4 + R) + samples S (R + (d+1) 4) + per vertex n (4 + R + (d+1) 4)
               (row offset, own row, one accumulator write)
      sampler  S x 32 (one probe sector per accepted sample; k-per-vertex forms)
      tiles    per tile P (R + (d+1) 4) (partner rows, partner accumulators)
      update   per vertex n ((d+1) 4 + 4d [+ 2d + 4d in the BF16 form]) (accumulator
               read, master write [, shadow write, master read])
    Returns {kernel: bytes, "epoch": total}."""
    R = position_row_bytes(d, precision)
    bf16 = bool(precision) and d >= 8
    acc = (d + 1) * 4
    out = {
        "sweep": 2 * m * (4 + R) + samples * (R + acc) + n * (4 + R + acc),
        "sampler": 32 * samples,
        "tiles": tiles * partners * (R + acc),
        "update": n * (acc + 4 * d + (6 * d if bf16 else 0)),
    }
    out["epoch"] = sum(out.values())
    return out


def tile_flops(tiles, d, partners=BLOCK_P, tile_vertices=BLOCK_T):
    """Floating-point operations of the block-sampled pairs: per pair and
    coordinate 3 for the squared distance (difference, square, add) and 2 each
    for the anchor and the partner term (Eq. 3's c (x_self - x_other))."""
    return tiles * tile_vertices * partners * 7 * d


def oriented_degrees(row_ptr, col_idx):
    """Out-degrees of the degree-oriented CSR the packed sweep (d <= 4, k
    samples per vertex) runs on: edge (i, j) belongs to i when
    (deg j, j) < (deg i, i), so each undirected edge appears once."""
    import numpy as np
    deg = np.diff(row_ptr).astype(np.int64)
    rows = np.repeat(np.arange(len(deg)), deg)
    ci = np.asarray(col_idx, dtype=np.int64)
    keep = (deg[ci] < deg[rows]) | ((deg[ci] == deg[rows]) & (ci < rows))
    return np.bincount(rows[keep], minlength=len(deg))


def sweep_algorithmic_bytes(n, nnz, d, k, n_units, accepted, oriented=False, row_bytes=None):
    """The implementation's own byte count of one sweep launch (what this
    design moves at least: work units, sample slots, a read-modify-write of
    every own and partner accumulator row, and in the oriented form the other
    endpoint's accumulator row per edge).  Reported beside the model of
    model_bytes, which is the roofline's numerator."""
    row = 4 * d if row_bytes is None else row_bytes
    acc_row = 4 * (((d + 1) + 3) // 4 * 4)
    common = 16 * n_units + 4 * n * k + n * row + n * 2 * acc_row + accepted * (row + 2 * acc_row)
    if oriented:
        m = nnz // 2
        return common + 8 * (n + 1) + 4 * m + m * (row + 2 * acc_row)
    return common + 4 * (n + 1) + 4 * nnz + nnz * row


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,utilization.gpu")

    def __init__(self, gpu_index, period_ms=20):
        self.gpu = gpu_index
        self.period_ms = period_ms
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", str(self.period_ms)], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        return self.parse(rows)

    @staticmethod
    def parse(rows):
        """Median SM clock over the samples taken under load (GPU utilisation
        above 0 where nvidia-smi reports it, else every sample), the maximum
        clock, and every throttle reason seen active."""
        num = re.compile(r"^[0-9.]+$")
        loaded = [r for r in rows if len(r) < 10 or not num.match(r[9]) or float(r[9]) > 0]
        sm = [float(r[1]) for r in (loaded or rows) if num.match(r[1])]
        mx = [float(r[2]) for r in rows if num.match(r[2])]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows), "samples_under_load": len(loaded)}


# ---------------------------------------------------------------------------
# CPU baseline: the oracle as it stands (OpenMP build over all host threads)
# ---------------------------------------------------------------------------
def oracle_epochs(w, epochs, x0=None, parallel=True, **form):
    """`epochs` oracle epochs of workload w from its initial positions (or
    x0); returns (pair-updates, seconds, positions)."""
    import oracle
    from paper_2011_03479_gb300 import inputs
    rp, ci = w["row_ptr"], w["col_idx"]
    n = len(rp) - 1
    x = oracle.init_positions(n, w["d"], inputs.EMBED_SEED) if x0 is None else x0
    m = len(ci) // 2
    t0 = time.perf_counter()
    xr, s, st = oracle.run(rp, ci, x, 1.0, epochs, inputs.EMBED_SEED, w["k"], parallel=parallel,
                           block_partners=form.get("block_partners", 0))
    dt = time.perf_counter() - t0
    return epochs * m + st["accepted"], dt, xr


def cpu_baseline(w, budget_s=12.0, **form):
    """The oracle on all host threads: one epoch to calibrate, then as many
    whole epochs as fit in the budget (at least one)."""
    import oracle
    threads = oracle.threads(parallel=True)
    p1, t1, _ = oracle_epochs(w, 1, **form)
    epochs = max(0, min(200, int(budget_s / max(t1, 1e-3)) - 1))
    p, t = p1, t1
    if epochs:
        p2, t2, _ = oracle_epochs(w, epochs, **form)
        p, t, epochs = p2, t2, epochs
    else:
        epochs = 1
    return {"value": p / t, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{epochs} whole epoch{'s' if epochs != 1 else ''} of {w['name']} from the initial "
                      f"positions, FP64 oracle (OpenMP build of the oracle's source), {threads} host threads"}


# ---------------------------------------------------------------------------
# ranks
# ---------------------------------------------------------------------------
def _dist():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return world, rank, local


def combine_ranks(t_total, pairs, device=None):
    """Whole-job figures over the ranks: the slowest rank's time and the sum
    of all ranks' pair-updates (one process per GPU, no data-path collective;
    this is the only exchange, after the timed region)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(t_total), float(pairs)
    tt = torch.tensor([float(t_total)], dtype=torch.float64, device=device)
    pp = torch.tensor([float(pairs)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    dist.all_reduce(pp, op=dist.ReduceOp.SUM)
    return tt.item(), pp.item()


def sum_ranks(value, device=None):
    """Sum of a per-rank rate over the ranks (the e2e figures)."""
    import torch
    import torch.distributed as dist
    if value is None or not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    v = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(v, op=dist.ReduceOp.SUM)
    return v.item()


def shard_jobs(sizes, world, rank):
    """Indices of the independent jobs (graphs of a batch) that rank `rank`
    of `world` takes: largest first, each to the rank with the least work so
    far (ties to the lower rank), so that every job is taken exactly once and
    the ranks' shares of the total size differ by at most the largest job."""
    load = [0] * world
    mine = []
    for q in sorted(range(len(sizes)), key=lambda q: (-sizes[q], q)):
        r = min(range(world), key=lambda r: (load[r], r))
        load[r] += sizes[q]
        if r == rank:
            mine.append(q)
    return sorted(mine)


def stream_share(n_jobs, world, rank):
    """Jobs of an arrival stream that rank `rank` serves: every world-th one."""
    return list(range(rank, n_jobs, world))


# ---------------------------------------------------------------------------
# profile summaries
# ---------------------------------------------------------------------------
PROFILE_TRAFFIC = {   # workload -> (summary under profiles/, key of the per-launch DRAM bytes of the timed kernel)
    "rmat-s16-ef16": ("sweep_rmat-s16-ef16.md", "traffic_bytes_per_launch"),
    "ba-n1m-m8": ("epoch_ba-n1m-m8.md", "traffic_bytes_per_launch_scaled"),
    "ba-n1m-m8-fp32": ("epoch_ba-n1m-m8-fp32.md", "traffic_bytes_per_launch_scaled"),
}


def _profile_traffic(kernel_src_hash, workload):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, if it was taken on the current kernel source (else None)."""
    if workload not in PROFILE_TRAFFIC:
        return None
    fname, key = PROFILE_TRAFFIC[workload]
    try:
        text = open(os.path.join(ROOT, "profiles", fname)).read()
    except OSError:
        return None
    m = re.search(key + r":\s*([0-9]+)", text)
    h = re.search(r"kernel_source_sha256:\s*([0-9a-f]+)", text)
    if not m or not h or h.group(1) != kernel_src_hash:
        return None
    return int(m.group(1))


# C-ABI front ends: host code that neither holds device code nor sets a launch
# shape, so a change there leaves the profiled kernels as they were
ABI_FRONT_ENDS = {"api.cu", "batch.cu", "serve.cu"}


def kernel_source_hash(csrc=None):
    """SHA-256 (first 16 hex digits) of the engine sources that define the
    kernels and their launch configuration: every .cu / .cuh of csrc but the
    C-ABI front ends.  A profile summary records it; its DRAM traffic is used
    only while the sources still hash the same."""
    hsh = hashlib.sha256()
    csrc = csrc or os.path.join(ROOT, "paper_2011_03479_gb300", "csrc")
    for fn in sorted(os.listdir(csrc)):
        if fn.endswith((".cu", ".cuh")) and fn not in ABI_FRONT_ENDS:
            hsh.update(open(os.path.join(csrc, fn), "rb").read())
    return hsh.hexdigest()[:16]


def _profile_key(workload, key):
    """A numeric key of the committed ncu summary of `workload` (e.g. the
    binding L1 / issue percentages), if taken on the current kernel source."""
    if workload not in PROFILE_TRAFFIC:
        return None
    try:
        text = open(os.path.join(ROOT, "profiles", PROFILE_TRAFFIC[workload][0])).read()
    except OSError:
        return None
    m = re.search(key + r":\s*([0-9.]+)", text)
    h = re.search(r"kernel_source_sha256:\s*([0-9a-f]+)", text)
    if not m or not h or h.group(1) != kernel_source_hash():
        return None
    return float(m.group(1))


# ---------------------------------------------------------------------------
# one graph: device-resident epochs, per-kernel windows, end-to-end jobs
# ---------------------------------------------------------------------------
def measure_single(w, form, steps, warmup, stream, flush, e2e_jobs=0, exact=False, shape=None):
    """Times `steps` epochs of workload w (after `warmup`) as gempe_step(ctx, 1),
    each bracketed by CUDA events on `stream` with an L2 flush before it;
    then as many epochs as gempe_sweep + gempe_update with the library's
    per-kernel events; then `e2e_jobs` whole jobs through the C ABI from
    pinned host memory."""
    import numpy as np
    import torch

    from paper_2011_03479_gb300 import binding as B
    from paper_2011_03479_gb300 import inputs

    rp, ci = w["row_ptr"], w["col_idx"]
    n, nnz, d, k = len(rp) - 1, len(ci), w["d"], w["k"]
    m = nnz // 2
    p = B.gempe_default_params(neg_per_vertex=k, seed=inputs.EMBED_SEED, **form)
    t0 = time.perf_counter()
    ctx = B.gempe_create(rp, ci, d, p, stream=stream)
    if shape:
        B.gempe_set_shape(ctx, **shape)
    stream.synchronize()
    create_s = time.perf_counter() - t0
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            flush.zero_()
            B.gempe_step(ctx, 1)
        torch.cuda.synchronize()
        s0 = B.gempe_stats(ctx)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for e0, e1 in ev:
            flush.zero_()          # L2 flush between steps, outside the events
            e0.record(stream)
            B.gempe_step(ctx, 1)
            e1.record(stream)
        torch.cuda.synchronize()
        s1 = B.gempe_stats(ctx)
        B.gempe_kernel_times(ctx, True)
        windows = []
        for _ in range(steps):
            flush.zero_()
            B.gempe_sweep(ctx)
            B.gempe_update(ctx)
            windows.append(B.gempe_kernel_times(ctx, True))
        B.gempe_kernel_times(ctx, False)
        torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    used = s1["used"] - s0["used"]             # sampled non-edges the timed epochs consumed
    draws = (s1["draws"] - s0["draws"]) * used / max(1, s1["accepted"] - s0["accepted"])
    pairs = steps * m + used
    rec = {"n": n, "m": m, "d": d, "k": k, "steps": steps, "pairs": pairs, "t_total": sum(step_ms) / 1e3,
           "ms_per_step": statistics.mean(step_ms), "ms_min": min(step_ms),
           "pairs_per_epoch": pairs / steps, "samples_per_epoch": used / steps, "draws_per_epoch": draws / steps,
           "kernel_ms": {"sweep": statistics.mean(x[0] for x in windows),
                         "tiles": statistics.mean(x[1] for x in windows),
                         "update": statistics.mean(x[2] for x in windows)},
           "sigma_fit_steps_last": s1["sigma_iters"], "create_s": create_s}
    if exact:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pe_exact, s_exact = B.gempe_loss_exact(ctx)
        dt = time.perf_counter() - t0
        rec["exact_pe"] = {"pairs_per_s": 0.5 * n * (n - 1) / dt, "ms": 1e3 * dt, "pe_bits": pe_exact,
                           "sigma": s_exact,
                           "how": "gempe_loss_exact(ctx, 0) once after the timed steps, host wall clock around the call"}
    ctx.close()
    if e2e_jobs > 0:
        rp_pin = torch.from_numpy(rp).pin_memory().numpy()
        ci_pin = torch.from_numpy(ci).pin_memory().numpy()
        out_pin = torch.empty((n, d), dtype=torch.float32).pin_memory().numpy()
        epochs = w["epochs"]

        def job():
            c = B.gempe_create(rp_pin, ci_pin, d, p, stream=stream)
            if shape:
                B.gempe_set_shape(c, **shape)
            B.gempe_step(c, epochs)
            B.gempe_positions(c, out_pin)
            u = B.gempe_stats(c)["used"]
            c.close()
            return epochs * m + u

        job()   # warm-up: the library is loaded, the pool holds memory, the GPU is warm
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_pairs = sum(job() for _ in range(e2e_jobs))
        torch.cuda.synchronize()
        e2e_t = max(time.perf_counter() - t0, 1e-9)
        rec["e2e"] = {"value": e2e_pairs / e2e_t, "unit": UNIT, "h2d_bytes_per_step": int(rp.nbytes + ci.nbytes),
                      "d2h_bytes_per_step": int(out_pin.nbytes),
                      "step": f"one {epochs}-epoch embedding job: gempe_create from pinned host CSR, "
                              f"gempe_step({epochs}), gempe_positions to pinned host memory",
                      "ms_per_job": 1e3 * e2e_t / e2e_jobs, "jobs": e2e_jobs}
    return rec


def roofline_of(rec, form, workload):
    """Per-kernel rooflines of one measured graph (model_bytes / tile_flops
    over the kernel's measured window) and the dominant kernel's record."""
    peak, peak_kind = _peaks()
    n, m, d = rec["n"], rec["m"], rec["d"]
    precision = form.get("precision", 0)
    block = bool(form.get("block_partners"))
    tiles = (n + BLOCK_T - 1) // BLOCK_T if block else 0
    samples = 0 if block else rec["samples_per_epoch"]
    mb = model_bytes(n, m, d, precision, samples, tiles)
    km = rec["kernel_ms"]
    kernels = {"sweep": {"bound": "hbm", "ms": km["sweep"], "algorithmic_bytes": mb["sweep"],
                         "achieved": mb["sweep"] / (km["sweep"] * 1e-3) / 1e9, "unit": "GB/s", "peak": peak}}
    kernels["sweep"]["frac"] = kernels["sweep"]["achieved"] / peak
    if block and km["tiles"] > 0:
        fl = tile_flops(tiles, d)
        if precision:
            from_peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
                if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
            tpk = float(from_peaks.get("bf16_tflops", 1900.0))
            kernels["tiles"] = {"bound": "tensor", "ms": km["tiles"], "algorithmic_flops": fl,
                                "achieved": fl / (km["tiles"] * 1e-3) / 1e12, "unit": "TFLOP/s", "peak": tpk,
                                "peak_kind": "measured cuBLAS bf16 burst" if from_peaks else "fallback bf16"}
        else:
            kernels["tiles"] = {"bound": "alu", "ms": km["tiles"], "algorithmic_flops": fl,
                                "achieved": fl / (km["tiles"] * 1e-3) / 1e12, "unit": "TFLOP/s",
                                "peak": FP32_PEAK_TFLOPS,
                                "peak_kind": "FP32 CUDA cores: 152 SMs x 128 lanes x 2 flops x 2.07 GHz"}
        kernels["tiles"]["frac"] = kernels["tiles"]["achieved"] / kernels["tiles"]["peak"]
        kernels["tiles"]["algorithmic_bytes"] = mb["tiles"]
    kernels["update"] = {"bound": "hbm", "ms": km["update"], "algorithmic_bytes": mb["update"],
                         "achieved": mb["update"] / max(km["update"] * 1e-3, 1e-12) / 1e9, "unit": "GB/s",
                         "peak": peak}
    kernels["update"]["frac"] = kernels["update"]["achieved"] / peak
    dom = max(kernels, key=lambda q: kernels[q]["ms"])
    kr = kernels[dom]
    names = {"sweep": "k_sweep", "update": "k_update",
             "tiles": "k_tile_tc (tcgen05)" if precision else "k_tile_f32"}
    roof = {"bound": kr["bound"], "kernel": names[dom], "achieved": kr["achieved"], "peak": kr["peak"],
            "unit": kr["unit"], "frac": kr["frac"],
            "peak_kind": kr.get("peak_kind", f"{peak_kind} HBM copy GB/s"),
            "traffic": _profile_traffic(kernel_source_hash(), workload) if dom == "sweep" else None,
            "algorithmic_per_launch": kr.get("algorithmic_bytes") if kr["unit"] == "GB/s" else kr["algorithmic_flops"],
            "window": "the kernel's mean window over the per-kernel pass (CUDA events on the launching stream)"}
    epoch_s = rec["ms_per_step"] * 1e-3
    model = {"bytes_per_epoch": mb["epoch"], "per_kernel_bytes": {q: mb[q] for q in ("sweep", "sampler", "tiles",
                                                                                     "update")},
             "achieved_gbs": mb["epoch"] / epoch_s / 1e9, "frac_of_hbm": mb["epoch"] / epoch_s / 1e9 / peak}
    return roof, kernels, model


# ---------------------------------------------------------------------------
# batched form: 256 SBM graphs, one CUDA-graph launch per epoch
# ---------------------------------------------------------------------------
def measure_batch(form, steps, warmup, stream, flush, world=1, rank=0, alone_steps=5, e2e=True, graphs=None):
    """This rank's share of the batch (shard_jobs by CSR size) as one batch:
    `steps` epochs as gempe_batch_step(b, 1) with CUDA events; then every
    graph of the share alone in its own plain FP32 context (alone_steps
    epochs each); then one whole batch job from pinned host memory."""
    import torch

    from paper_2011_03479_gb300 import binding as B
    from paper_2011_03479_gb300 import inputs

    w = inputs.sbm_batch_256() if graphs is None else graphs
    all_graphs, k = w["graphs"], w["k"]
    share = shard_jobs([len(g["col_idx"]) + len(g["row_ptr"]) for g in all_graphs], world, rank)
    graphs = [all_graphs[q] for q in share]
    G = len(graphs)
    p = B.gempe_default_params(neg_per_vertex=k, seed=inputs.EMBED_SEED, **form)
    desc = [(g["row_ptr"], g["col_idx"], g["d"]) for g in graphs]
    m_tot = sum(len(g["col_idx"]) // 2 for g in graphs)
    n_tot = sum(len(g["row_ptr"]) - 1 for g in graphs)
    t0 = time.perf_counter()
    b = B.gempe_batch_create(desc, p, stream=stream)
    create_s = time.perf_counter() - t0
    dims = sorted({g["d"] for g in graphs})
    shapes = {d: B.gempe_batch_shape(b, d) for d in dims}
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            flush.zero_()
            B.gempe_batch_step(b, 1)
        torch.cuda.synchronize()
        used0 = sum(B.gempe_batch_stats(b, q)["used"] for q in range(G))
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for e0, e1 in ev:
            flush.zero_()
            e0.record(stream)
            B.gempe_batch_step(b, 1)
            e1.record(stream)
        torch.cuda.synchronize()
        used = sum(B.gempe_batch_stats(b, q)["used"] for q in range(G)) - used0
    b.close()
    step_ms = [a.elapsed_time(c) for a, c in ev]
    pairs = steps * m_tot + used
    rec = {"graphs": G, "n_total": n_tot, "m_total": m_tot, "dims": {str(d): sum(1 for g in graphs if g["d"] == d)
                                                                     for d in dims},
           "pairs": pairs, "t_total": sum(step_ms) / 1e3, "ms_per_step": statistics.mean(step_ms),
           "pairs_per_epoch": pairs / steps, "samples_per_epoch": used / steps, "create_s": create_s,
           "shapes": {str(d): sh for d, sh in shapes.items()}}
    # the plain form: every graph in its own FP32 context, one after the other
    if alone_steps:
        alone_pairs, alone_s = 0, 0.0
        pa = B.gempe_default_params(neg_per_vertex=k)
        ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for q, g in zip(share, graphs):
            pa.seed = inputs.EMBED_SEED ^ q
            c = B.gempe_create(g["row_ptr"], g["col_idx"], g["d"], pa, stream=stream)
            with torch.cuda.stream(stream):
                B.gempe_step(c, 1)          # captures the epoch graph
                u0 = B.gempe_stats(c)["used"]
                flush.zero_()
                ea.record(stream)
                B.gempe_step(c, alone_steps)
                eb.record(stream)
                eb.synchronize()
            alone_s += ea.elapsed_time(eb) / 1e3
            alone_pairs += alone_steps * (len(g["col_idx"]) // 2) + B.gempe_stats(c)["used"] - u0
            c.close()
        rec["alone_fp32"] = {"pairs": alone_pairs, "t": alone_s, "steps": alone_steps}
    if e2e:
        epochs = w["epochs"]
        pinned = [(torch.from_numpy(g["row_ptr"]).pin_memory().numpy(),
                   torch.from_numpy(g["col_idx"]).pin_memory().numpy(), g["d"]) for g in graphs]
        h2d = sum(a.nbytes + c.nbytes for a, c, _ in pinned)
        d2h = sum(4 * (len(a) - 1) * d for a, _, d in pinned)
        outs = [torch.empty((len(a) - 1, d), dtype=torch.float32).pin_memory().numpy() for a, _, d in pinned]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        jb = B.gempe_batch_create(pinned, p, stream=stream)
        B.gempe_batch_step(jb, epochs)
        for q in range(G):
            B.gempe_batch_positions(jb, q, outs[q])
        e2e_pairs = epochs * m_tot + sum(B.gempe_batch_stats(jb, q)["used"] for q in range(G))
        jb.close()
        e2e_t = time.perf_counter() - t0
        rec["e2e"] = {"value": e2e_pairs / e2e_t, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                      "d2h_bytes_per_step": int(d2h),
                      "step": f"one batch job: gempe_batch_create of {G} graphs from pinned host CSR (host "
                              f"validation included), gempe_batch_step({epochs}), gempe_batch_positions of every "
                              f"graph into pinned memory", "ms_per_job": 1e3 * e2e_t}
    # algorithmic bytes of one epoch (model_bytes of every graph)
    byts = 0.0
    for g in graphs:
        n_g, m_g, d = len(g["row_ptr"]) - 1, len(g["col_idx"]) // 2, g["d"]
        byts += model_bytes(n_g, m_g, d, form.get("precision", 0), used / steps * (n_g / n_tot))["epoch"]
    rec["bytes_per_epoch"] = byts
    return rec


# ---------------------------------------------------------------------------
# served form: Poisson arrivals of R-MAT jobs
# ---------------------------------------------------------------------------
def measure_serve(form, n_jobs, warmup, world=1, rank=0, cap_jobs=100, rate=50.0):
    """n_jobs jobs arrive as a Poisson stream (mean `rate` per second): each an
    R-MAT graph with scale uniform in 10..18 and edge factor uniform in 8..16
    (a pool of two graphs per scale, generated before the timed region), d
    from {2, 32, 128}, 100-300 epochs, k = 10, its own seed.  This rank
    serves every world-th job of the stream (stream_share) through
    gempe_server_submit at its arrival time, on a server with a 120 GB budget
    and 32 job slots; then the first cap_jobs of its jobs again, all at once
    (the capacity)."""
    import numpy as np
    import torch

    from paper_2011_03479_gb300 import binding as B
    from paper_2011_03479_gb300 import inputs

    rng = np.random.default_rng(5000)
    pool = {}
    for scale in range(10, 19):
        pool[scale] = []
        for r in range(2):
            ef = int(rng.integers(8, 17))
            rp, ci = inputs.rmat(scale, ef, seed=5001 + 100 * scale + r)
            pool[scale].append((rp, ci, ef))
    k = 10
    budget = 120 * (1 << 30)
    p = B.gempe_default_params(neg_per_vertex=k, seed=inputs.EMBED_SEED, **form)

    def draw_job(q):
        scale = int(rng.integers(10, 19))
        rp, ci, ef = pool[scale][int(rng.integers(0, 2))]
        return dict(rp=rp, ci=ci, d=int(rng.choice([2, 32, 128])), epochs=int(rng.integers(100, 301)),
                    seed=inputs.EMBED_SEED ^ (q + 1), scale=scale, ef=ef)

    stream_jobs = [draw_job(q) for q in range(n_jobs)]
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n_jobs))
    mine = stream_share(n_jobs, world, rank)
    srv = B.gempe_server_create(budget, max_jobs=32, params=p)
    for q in range(warmup):
        j = stream_jobs[q % n_jobs]
        jid = B.gempe_server_submit(srv, j["rp"], j["ci"], j["d"], 20, j["seed"] ^ 0x5A5A)
        B.gempe_server_wait(srv, jid, 600000)
        B.gempe_server_result(srv, jid)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ids = []
    for q in mine:
        j = stream_jobs[q]
        dt = arrivals[q] - (time.perf_counter() - t0)
        if dt > 0:
            time.sleep(dt)
        ids.append(B.gempe_server_submit(srv, j["rp"], j["ci"], j["d"], j["epochs"], j["seed"]))
    infos = [B.gempe_server_wait(srv, i, 3600 * 1000) for i in ids]
    wall = time.perf_counter() - t0
    for i in ids:
        B.gempe_server_result(srv, i)
    stats = B.gempe_server_stats(srv)
    cap = [stream_jobs[q] for q in mine[:cap_jobs]]
    cids = [B.gempe_server_submit(srv, j["rp"], j["ci"], j["d"], j["epochs"], j["seed"]) for j in cap]
    cinfos = [B.gempe_server_wait(srv, i, 3600 * 1000) for i in cids]
    for i in cids:
        B.gempe_server_result(srv, i)
    srv.close()
    cap_span = (max(c["done_ns"] for c in cinfos) - min(c["submit_ns"] for c in cinfos)) / 1e9
    sub = np.array([inf["submit_ns"] for inf in infos], dtype=np.float64)
    adm = np.array([inf["admit_ns"] for inf in infos], dtype=np.float64)
    done = np.array([inf["done_ns"] for inf in infos], dtype=np.float64)
    lat = (done - sub) / 1e6
    wait = (adm - sub) / 1e6
    pairs = float(sum(inf["pairs"] for inf in infos))
    span = (done.max() - sub.min()) / 1e9
    my_jobs = [stream_jobs[q] for q in mine]
    return {"jobs": len(mine), "stream_jobs": n_jobs, "pairs": pairs, "span_s": span, "wall_s": wall,
            "value": pairs / span,
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "mean": float(lat.mean()), "max": float(lat.max())},
            "queue_wait_ms": {"p50": float(np.percentile(wait, 50)), "p99": float(np.percentile(wait, 99))},
            "offered_pairs_per_s": pairs / max((sub.max() - sub.min()) / 1e9, 1e-9),
            "capacity_pairs_per_s": sum(c["pairs"] for c in cinfos) / cap_span,
            "capacity_jobs": len(cap),
            "peak_device_bytes": stats["peak_bytes_in_use"], "failed_jobs": stats["failed"],
            "h2d_bytes_per_job": float(np.mean([j["rp"].nbytes + j["ci"].nbytes for j in my_jobs])),
            "d2h_bytes_per_job": float(np.mean([4 * (len(j["rp"]) - 1) * j["d"] for j in my_jobs])),
            "gpu_launches": int(sum(3 + (5 if j["d"] <= 4 else 0) + 3 * j["epochs"] for j in my_jobs))}


# ---------------------------------------------------------------------------
# the headline line
# ---------------------------------------------------------------------------
def _setup():
    import torch
    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    return world, rank, local, dev, stream, flush


def _finish(world):
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _nested_single(workload, w, args, stream, flush, dev):
    form = FORMS[workload]
    steps = max(args.steps, 100)    # 44 us epochs: enough of them for stable events
    rec = measure_single(w, form, steps, args.warmup, stream, flush, e2e_jobs=1, exact=True)
    t, p = combine_ranks(rec["t_total"], rec["pairs"], dev)
    roof, kernels, model = roofline_of(rec, form, workload)
    l1 = _profile_key(workload, "binding_l1_pct")
    issue = _profile_key(workload, "binding_issue_active_pct")
    roof["binding"] = {"l1_throughput_pct": l1, "issue_active_pct": issue,
                       "note": "the graph's working set stays in L2 (the sweep reads about 9 MB of DRAM per launch "
                               "after the flush), so the HBM fraction understates it; these ncu counters of the "
                               "committed profile summary show what binds (None: profile not of the current source)"}
    e2e = rec.get("e2e")
    if e2e:
        e2e = dict(e2e, value=sum_ranks(e2e["value"], dev))
    return {"value": p / t, "unit": UNIT, "dtype": "f32", "ms_per_step": rec["ms_per_step"], "steps": steps,
            "config": {"workload": workload, "n": rec["n"], "m": rec["m"], "d": rec["d"],
                       "sampling": f"k={rec['k']} per vertex", "sigma_every": 1},
            "pairs_per_epoch": rec["pairs_per_epoch"], "kernel_ms": rec["kernel_ms"], "roofline": roof,
            "kernels": kernels, "epoch_model": model, "e2e": e2e, "exact_pe": rec.get("exact_pe"),
            "gpu_launches": 3 * 2 * steps}


def _nested_batch(args, stream, flush, dev, world, rank):
    out = {}
    from paper_2011_03479_gb300 import inputs
    graphs = inputs.sbm_batch_256()
    for name in ("sbm-batch-256", "sbm-batch-256-bf16"):
        form = FORMS[name]
        bf16 = bool(form.get("precision"))
        rec = measure_batch(form, args.steps, args.warmup, stream, flush, world, rank,
                            alone_steps=0 if bf16 else 5, e2e=not bf16, graphs=graphs)
        t, p = combine_ranks(rec["t_total"], rec["pairs"], dev)
        r = {"value": p / t, "unit": UNIT, "dtype": "bf16 positions (d >= 8), f32 sums" if bf16 else "f32",
             "ms_per_step": rec["ms_per_step"], "steps": args.steps,
             "config": {"workload": name, "graphs": rec["graphs"], "n_total": rec["n_total"],
                        "m_total": rec["m_total"], "dims": rec["dims"], "k": 5,
                        "share": f"rank {rank} of {world}: graphs by CSR size, largest first to the least loaded rank"},
             "pairs_per_epoch": rec["pairs_per_epoch"], "shapes": rec["shapes"], "create_s": rec["create_s"],
             "epoch_model": {"bytes_per_epoch": rec["bytes_per_epoch"],
                             "frac_of_hbm": rec["bytes_per_epoch"] / (rec["ms_per_step"] * 1e-3) / 1e9 / _peaks()[0]},
             "gpu_launches": args.steps * 3 * len(rec["dims"])}
        if "alone_fp32" in rec:
            ta, pa = combine_ranks(rec["alone_fp32"]["t"], rec["alone_fp32"]["pairs"], dev)
            r["alone_fp32"] = {"value": pa / ta, "unit": UNIT, "ratio": (p / t) / (pa / ta),
                               "how": f"each graph of the share in its own FP32 context (gempe_create + gempe_step), "
                                      f"one after the other, {rec['alone_fp32']['steps']} epochs each, CUDA events "
                                      f"around each graph's epochs"}
        if rec.get("e2e"):
            r["e2e"] = dict(rec["e2e"], value=sum_ranks(rec["e2e"]["value"], dev))
        out[name] = r
    fp, bf = out["sbm-batch-256"], out["sbm-batch-256-bf16"]
    fp["vs_plain_fp32"] = {"bf16_form": bf["value"] / fp["value"],
                           "batched_vs_alone": fp.get("alone_fp32", {}).get("ratio")}
    return out


def _nested_serve(args, dev, world, rank):
    out = {}
    for name in ("rmat-serve-poisson50", "rmat-serve-poisson50-bf16"):
        form = FORMS[name]
        bf16 = bool(form.get("precision"))
        rec = measure_serve(form, args.serve_jobs, 2, world, rank, cap_jobs=min(100, args.serve_jobs))
        out[name] = {"value": sum_ranks(rec["value"], dev), "unit": UNIT,
                     "dtype": "bf16 positions (d >= 8), f32 sums" if bf16 else "f32",
                     "config": {"workload": name, "jobs": rec["jobs"], "stream_jobs": rec["stream_jobs"],
                                "arrival_rate_per_s": 50, "scale": "U{10..18}", "edge_factor": "U{8..16}",
                                "d": [2, 32, 128], "epochs": "U{100..300}", "k": 10, "budget_bytes": 120 << 30,
                                "max_jobs": 32, "share": f"every {world}th job of the stream from job {rank}"},
                     "latency_ms": rec["latency_ms"], "queue_wait_ms": rec["queue_wait_ms"],
                     "offered_pairs_per_s": rec["offered_pairs_per_s"],
                     "capacity_pairs_per_s": rec["capacity_pairs_per_s"],
                     "capacity_note": f"{rec['capacity_jobs']} of the same jobs submitted at once; when the offered "
                                      "load is above this the latency is dominated by the queue",
                     "peak_device_bytes": rec["peak_device_bytes"], "failed_jobs": rec["failed_jobs"],
                     "e2e": {"value": sum_ranks(rec["value"], dev), "unit": UNIT,
                             "h2d_bytes_per_step": int(rec["h2d_bytes_per_job"]),
                             "d2h_bytes_per_step": int(rec["d2h_bytes_per_job"]),
                             "step": "one job: arrival to positions on the host (gempe_server_submit .. "
                                     "gempe_server_result)"},
                     "gpu_launches": rec["gpu_launches"]}
    out["rmat-serve-poisson50"]["vs_plain_fp32"] = {
        "bf16_form_capacity": out["rmat-serve-poisson50-bf16"]["capacity_pairs_per_s"] /
        out["rmat-serve-poisson50"]["capacity_pairs_per_s"]}
    return out


def run_headline(args):
    from paper_2011_03479_gb300 import inputs
    world, rank, local, dev, stream, flush = _setup()
    w = inputs.ba_1m()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    wall0 = time.perf_counter()
    fp32 = measure_single(w, FORMS["ba-n1m-m8-fp32"], args.steps, args.warmup, stream, flush, e2e_jobs=args.e2e_jobs)
    bf16 = measure_single(w, FORMS["ba-n1m-m8"], args.steps, args.warmup, stream, flush, e2e_jobs=args.e2e_jobs)
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    t, p = combine_ranks(fp32["t_total"], fp32["pairs"], dev)
    value = p / t
    tb, pb = combine_ranks(bf16["t_total"], bf16["pairs"], dev)
    bf_value = pb / tb
    roof, kernels, model = roofline_of(fp32, FORMS["ba-n1m-m8-fp32"], "ba-n1m-m8-fp32")
    roof_b, kernels_b, model_b = roofline_of(bf16, FORMS["ba-n1m-m8"], "ba-n1m-m8")
    e2e = fp32.get("e2e")
    if e2e:
        e2e = dict(e2e, value=sum_ranks(e2e["value"], dev))
    e2e_b = bf16.get("e2e")
    if e2e_b:
        e2e_b = dict(e2e_b, value=sum_ranks(e2e_b["value"], dev))
    nested = {}
    if not args.no_nested:
        nested["rmat-s16-ef16"] = _nested_single("rmat-s16-ef16", inputs.rmat_s16(), args, stream, flush, dev)
        nested.update(_nested_batch(args, stream, flush, dev, world, rank))
        nested.update(_nested_serve(args, dev, world, rank))
    if rank != 0:
        _finish(world)
        return
    per_epoch_launches = 4      # sweep, tiles, update, and the next epoch's block sampler (side stream)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": fp32["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": HEADLINE, "n": fp32["n"], "m": fp32["m"], "d": fp32["d"],
                   "sampling": "block 128x64 (every tile of 128 vertices meets 64 partners per epoch)",
                   "precision": "plain FP32: FP32 positions, FP32 pair arithmetic and sums",
                   "sigma_every": 1, "epochs_per_job": w["epochs"],
                   "step": "one epoch: gempe_step(ctx, 1), a replay of the captured epoch graph",
                   "l2": "flushed between steps (256 MiB write outside the timed events)",
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
        "pairs_per_epoch": fp32["pairs_per_epoch"],
        "kernel_ms": fp32["kernel_ms"],
        "bf16_form": {"value": bf_value, "unit": UNIT, "ms_per_step": bf16["ms_per_step"],
                      "dtype": "bf16 positions (tcgen05 tiles), f32 master positions and sums",
                      "pairs_per_epoch": bf16["pairs_per_epoch"], "kernel_ms": bf16["kernel_ms"],
                      "roofline": roof_b, "kernels": kernels_b, "epoch_model": model_b, "e2e": e2e_b,
                      "how": "the same seed and graph, own context, same steps, warm-up and flushes, CUDA events"},
        "vs_plain_fp32": {"bf16_form": bf_value / value,
                          "bf16_form_e2e": (e2e_b["value"] / e2e["value"]) if (e2e and e2e_b) else None},
        "roofline": roof,
        "kernels": kernels,
        "epoch_model": model,
        "clocks": clk,
        "e2e": e2e,
        "gpu_launches": per_epoch_launches * 2 * args.steps,
        "gpu_launches_note": "the FP32 line's timed passes (value pass and per-kernel pass): per epoch the sweep, "
                             "the FP32 tiles, the update and the next epoch's block sampler",
        "wall_s_timed_region": wall,
        "nested": nested,
    }
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(dict(w, name=HEADLINE), budget_s=args.cpu_budget,
                                            block_partners=BLOCK_P)
    print(json.dumps(line))
    _finish(world)


def run_workload(args):
    """One workload alone (the profiling commands use these lines)."""
    from paper_2011_03479_gb300 import inputs
    world, rank, local, dev, stream, flush = _setup()
    name = args.workload
    clocks = ClockSampler(local)
    clocks.start()
    if name in BATCH_WORKLOADS:
        rec = measure_batch(FORMS[name], args.steps, args.warmup, stream, flush, world, rank,
                            alone_steps=0, e2e=args.e2e_jobs > 0)
        t, p = combine_ranks(rec["t_total"], rec["pairs"], dev)
        line = {"value": p / t, "ms_per_step": rec["ms_per_step"], "config": {"workload": name}, "record": rec}
    elif name in SERVE_WORKLOADS:
        rec = measure_serve(FORMS[name], args.serve_jobs, args.warmup, world, rank)
        line = {"value": sum_ranks(rec["value"], dev), "ms_per_step": None, "config": {"workload": name},
                "record": rec}
    else:
        w = inputs.WORKLOADS[name.replace("-fp32", "")]()
        rec = measure_single(w, FORMS[name], args.steps, args.warmup, stream, flush, e2e_jobs=args.e2e_jobs)
        t, p = combine_ranks(rec["t_total"], rec["pairs"], dev)
        roof, kernels, model = roofline_of(rec, FORMS[name], name)
        line = {"value": p / t, "ms_per_step": rec["ms_per_step"], "config": {"workload": name, "n": rec["n"],
                                                                              "m": rec["m"], "d": rec["d"]},
                "kernel_ms": rec["kernel_ms"], "roofline": roof, "kernels": kernels, "epoch_model": model,
                "pairs_per_epoch": rec["pairs_per_epoch"], "e2e": rec.get("e2e")}
    clk = clocks.stop()
    if rank == 0:
        line.update({"metric": METRIC, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                     "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "data": "synthetic",
                     "clocks": clk})
        print(json.dumps(line))
    _finish(world)


# ---------------------------------------------------------------------------
# reference arm: the oracle on the host cores
# ---------------------------------------------------------------------------
REF_SAMPLE_N = 62500     # the headline's generator at 1/16 of its vertices: same m, d and tiles


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_2011_03479_gb300 import inputs
    oracle.build()
    threads = oracle.threads(parallel=True)
    rp, ci = inputs.barabasi_albert(REF_SAMPLE_N, 8, seed=3001)
    w = {"name": f"ba-n{REF_SAMPLE_N}-m8", "row_ptr": rp, "col_idx": ci, "d": 64, "k": 0}
    m = len(ci) // 2
    x = None
    if args.warmup:
        _, _, x = oracle_epochs(w, args.warmup, block_partners=BLOCK_P)
    times, pairs = [], 0
    for s in range(args.steps):
        p, t, x = oracle_epochs(w, 1, x0=x, block_partners=BLOCK_P)
        times.append(t)
        pairs += p
    value = pairs / sum(times)
    sample = (f"one FP64 oracle epoch per step (OpenMP build, {threads} host threads) of a Barabasi-Albert graph "
              f"with n = {REF_SAMPLE_N}, m = 8 (the headline's generator at 1/16 of its vertices, {m} edges), "
              f"d = 64, block sampling 128 x 64: the same work per pair as {HEADLINE}")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": HEADLINE, "n": 1000000, "m": "~8.0e6", "d": 64,
                   "sampling": "block 128x64 (every tile of 128 vertices meets 64 partners per epoch)",
                   "step": "one epoch of the FP64 CPU oracle on a bounded sample of the workload"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["gempe", "reference"], default="gempe")
    ap.add_argument("--e2e-jobs", type=int, default=1)
    ap.add_argument("--serve-jobs", type=int, default=200, help="jobs of each serving run (at 50 per second)")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-nested", action="store_true",
                    help="the headline workload only (no graph-drawing, batched or served records)")
    ap.add_argument("--workload", choices=sorted(FORMS), default=None,
                    help="one workload alone instead of the headline line")
    args = ap.parse_args()
    if args.impl == "reference":
        if args.steps > 50:
            args.steps = 50      # each oracle step takes a fraction of a second: keep the run bounded
        run_reference(args)
    elif args.workload:
        run_workload(args)
    else:
        run_headline(args)


if __name__ == "__main__":
    main()
