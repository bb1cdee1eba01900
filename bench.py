#!/usr/bin/env python3
"""GEMPE epoch benchmark: pair-updates per second of one GEMPE epoch.

Workload (default): the graph-drawing-at-scale setting -- an R-MAT graph with
scale 16 (65,536 vertices) and edge factor 16 ((a,b,c,d) = (.57,.19,.19,.05),
duplicates and self loops removed), d = 2 FP32 positions, 10 sampled non-edges
per vertex per epoch, sigma refit after every epoch.  Synthetic, seeded.

A step is one epoch (pair sweep + position update + sigma refit) through the
C ABI (gempe_step(ctx, 1): one replay of the captured epoch graph) on a torch
CUDA stream.  Each step is timed with CUDA events on that stream; the L2
cache is flushed (a 256 MiB write) between steps, outside the events.  A
second pass of as many epochs, split as gempe_sweep / event / gempe_update,
gives the sweep kernel's window for the roofline line.  Pair-updates per
epoch = m undirected edges + accepted sampled non-edges.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gempe|reference]

--impl reference times the FP64 CPU oracle (the method restated in plain C,
single-threaded) on the same workload and metric: each step is one oracle
epoch.  Under torchrun (N > 1) every rank runs an independent replica of the
workload on its own GPU (no collective on the data path); value is the sum of
all ranks' pair-updates over the slowest rank's time.
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

METRIC = "pair-updates/sec per GEMPE epoch"
UNIT = "pair-updates/s"
WORKLOAD = "rmat-s16-ef16"
# engine parameters of each workload (the graph and d, k come from inputs.WORKLOADS)
FORMS = {
    "rmat-s16-ef16": {},
    "ba-n1m-m8": {"block_partners": 64, "precision": 1},          # BF16 + tensor-core tiles
    "ba-n1m-m8-fp32": {"block_partners": 64, "precision": 0},     # the plain FP32 run of the same seed
    "ba-n300k-m8": {"block_partners": 64, "precision": 1},        # the same kernels at a size for full ncu captures
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
EDGE_CHUNK = 64      # CSR slots per work unit of the d >= 8 sweep
UNIT_PAIRS = 128     # edge + sample slots per packed work unit of the d <= 4 sweep


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


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


def position_row_bytes(d, precision):
    """Bytes of the position row the pair arithmetic reads: the BF16 shadow
    (2d) in the precision form (d >= 8), else the FP32 positions (4d)."""
    return 2 * d if precision and d >= 8 else 4 * d


def sweep_algorithmic_bytes(n, nnz, d, k, n_units, accepted, oriented=False, row_bytes=None):
    """Bytes one sweep launch must move at least, each random gather paid once
    at its minimum size (no reuse): CSR streamed once, work units, the sample
    slots, own row, a read-modify-write of every own accumulator row, the
    partner row and a read-modify-write of the partner's accumulator row per
    accepted sample, and per edge slot the neighbour's row -- once per CSR
    slot when each endpoint sums its own edges, or (oriented form) once per
    undirected edge plus the read-modify-write of the other endpoint's
    accumulator row, with the full row offsets read for the degrees.  A row
    is row_bytes (position_row_bytes: 4d FP32, 2d for BF16 positions)."""
    row = 4 * d if row_bytes is None else row_bytes
    acc_row = 4 * (((d + 1) + 3) // 4 * 4)
    common = 16 * n_units + 4 * n * k + n * row + n * 2 * acc_row + accepted * (row + 2 * acc_row)
    if oriented:
        m = nnz // 2
        return common + 8 * (n + 1) + 4 * m + m * (row + 2 * acc_row)
    return common + 4 * (n + 1) + 4 * nnz + nnz * row


def tile_algorithmic_bytes(n, d, n_tiles, partners=64):
    """Block-sampled non-edges on the tensor-core tiles: every vertex's BF16 row
    and mask once, every tile's partner rows, a read-modify-write of every
    anchor's and every partner's accumulator row."""
    acc_row = 4 * (((d + 1) + 3) // 4 * 4)
    return n * (2 * d + 8 + 2 * acc_row) + n_tiles * partners * (4 + 2 * d + 2 * acc_row)


def sampler_algorithmic_bytes(n, k, draws):
    """One 32-byte hash-set sector per draw and the 4-byte partner per slot."""
    return 32 * draws + 4 * n * k


def work_units(row_ptr, k, d, edge_chunk=EDGE_CHUNK, unit_pairs=UNIT_PAIRS, out_degrees=None, kernel=0):
    """Number of sweep work units (mirrors the library's unit building: d >= 8
    or kernel 1, chunks of each vertex's row; d <= 4 packed units, over the
    oriented CSR's out-degrees when they are given)."""
    import numpy as np
    deg = np.diff(row_ptr).astype(np.int64)
    if d > 4 or kernel == 1:
        return int(np.maximum(1, (deg + edge_chunk - 1) // edge_chunk).sum())
    if out_degrees is not None:
        deg = np.asarray(out_degrees, dtype=np.int64)
    units, i, n = 0, 0, len(deg)
    pairs = deg + k
    while i < n:
        if pairs[i] > unit_pairs:
            units += int((deg[i] - 1) // unit_pairs) + 1 if deg[i] > unit_pairs else 1
            i += 1
            continue
        v0, tot = i, 0
        while i < n and i - v0 < 32 and pairs[i] <= unit_pairs and tot + pairs[i] <= unit_pairs:
            tot += pairs[i]
            i += 1
        units += 1
    return units


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
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
        sm = [float(r[1]) for r in rows if re.match(r"^[0-9.]+$", r[1])]
        mx = [float(r[2]) for r in rows if re.match(r"^[0-9.]+$", r[2])]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# ---------------------------------------------------------------------------
# CPU baseline: the oracle as it stands, single-threaded, bounded sample
# ---------------------------------------------------------------------------
def oracle_epochs(w, epochs, x0=None):
    import numpy as np
    import oracle
    rp, ci = w["row_ptr"], w["col_idx"]
    n = len(rp) - 1
    from paper_2011_03479_gb300 import inputs
    x = oracle.init_positions(n, w["d"], inputs.EMBED_SEED) if x0 is None else x0
    m = len(ci) // 2
    t0 = time.perf_counter()
    xr, s, st = oracle.run(rp, ci, x, 1.0, epochs, inputs.EMBED_SEED, w["k"])
    dt = time.perf_counter() - t0
    return epochs * m + st["accepted"], dt, xr


def cpu_baseline(w, budget_s=12.0):
    # calibrate on one epoch, then run as many as fit in the budget
    p1, t1, _ = oracle_epochs(w, 1)
    epochs = max(1, min(200, int(budget_s / max(t1, 1e-3))))
    p, t, _ = oracle_epochs(w, epochs)
    return {"value": p / t, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{epochs} epoch{'s' if epochs != 1 else ''} of {w['name']} from the initial positions, "
                      "FP64 oracle, one thread"}


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


PROFILE_TRAFFIC = {   # workload -> (summary under profiles/, key of the per-launch DRAM bytes of the timed kernel)
    "rmat-s16-ef16": ("sweep_rmat-s16-ef16.md", "traffic_bytes_per_launch"),
    "ba-n1m-m8": ("epoch_ba-n1m-m8.md", "traffic_bytes_per_launch_scaled"),
}


def combine_ranks(t_total, pairs, device=None):
    """Whole-job figures over the replicas: the slowest rank's time and the sum
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
    """Sum of a per-rank rate over the replicas (the e2e figures)."""
    import torch
    import torch.distributed as dist
    if value is None or not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    v = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(v, op=dist.ReduceOp.SUM)
    return v.item()


def _profile_traffic(kernel_src_hash, workload=WORKLOAD):
    """DRAM bytes per sweep launch from the committed ncu summary, if it was
    taken on the current kernel source (else None)."""
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


def run_gempe(args):
    import numpy as np
    import torch

    from paper_2011_03479_gb300 import binding as B
    from paper_2011_03479_gb300 import inputs

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    workload = args.workload
    w = inputs.WORKLOADS[workload.replace("-fp32", "")]()
    rp, ci = w["row_ptr"], w["col_idx"]
    n, nnz, d, k = len(rp) - 1, len(ci), w["d"], w["k"]
    m = nnz // 2
    form = FORMS[workload]
    p = B.gempe_default_params(neg_per_vertex=k, seed=inputs.EMBED_SEED, **form)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    # ---------------- device-resident timing ----------------
    # Pass A (the value): each step is one epoch as a user runs it,
    # gempe_step(ctx, 1), a replay of the captured epoch graph.  Pass B (the
    # sweep kernel's window for the roofline): the same number of epochs
    # split at the sweep, gempe_sweep / event / gempe_update; the event
    # between them makes the update wait for the whole sweep, so these steps
    # are slower and only their sweep window is used.
    def timed_events(k, split):
        return [tuple(torch.cuda.Event(enable_timing=True) for _ in range(3 if split else 2)) for _ in range(k)]

    ctx = B.gempe_create(rp, ci, d, p, stream=stream)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush.zero_()
            B.gempe_step(ctx, 1)
        for _ in range(args.warmup):
            flush.zero_()
            B.gempe_sweep(ctx)
            B.gempe_update(ctx)
        torch.cuda.synchronize()
        s0 = B.gempe_stats(ctx)
        ev = timed_events(args.steps, False)
        ev_split = timed_events(args.steps, True)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        clocks = ClockSampler(local)
        clocks.start()
        wall0 = time.perf_counter()
        for e0, e2 in ev:
            flush.zero_()          # L2 flush between steps, outside the events
            e0.record(stream)
            B.gempe_step(ctx, 1)
            e2.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
        s1 = B.gempe_stats(ctx)
        for e0, e1, e2 in ev_split:
            flush.zero_()
            e0.record(stream)
            B.gempe_sweep(ctx)
            e1.record(stream)
            B.gempe_update(ctx)
            e2.record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
    step_ms = [a.elapsed_time(c) for a, c in ev]
    sweep_ms = [a.elapsed_time(b) for a, b, c in ev_split]
    split_ms = [a.elapsed_time(c) for a, b, c in ev_split]
    accepted = s1["used"] - s0["used"]          # sampled non-edges the timed sweeps consumed
    draws = (s1["draws"] - s0["draws"]) * accepted / max(1, s1["accepted"] - s0["accepted"])
    pairs = args.steps * m + accepted
    t_total = sum(step_ms) / 1e3
    t_all, pairs_all = combine_ranks(t_total, pairs, dev)
    value = pairs_all / t_all
    # the exact Eq. 2 over all n(n-1)/2 pairs (on demand, not part of an epoch)
    exact = None
    if n <= 131072:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pe_exact, s_exact = B.gempe_loss_exact(ctx)
        dt = time.perf_counter() - t0
        exact = {"pairs_per_s": 0.5 * n * (n - 1) / dt, "ms": 1e3 * dt, "pe_bits": pe_exact, "sigma": s_exact,
                 "how": "gempe_loss_exact(ctx, 0) once after the timed steps, host wall clock around the call"}
    ctx.close()

    # ---------------- end to end through the C ABI, host buffers ----------------
    rp_pin = torch.from_numpy(rp).pin_memory().numpy()
    ci_pin = torch.from_numpy(ci).pin_memory().numpy()
    out_pin = torch.empty((n, d), dtype=torch.float32).pin_memory().numpy()
    epochs = w["epochs"]
    e2e_jobs = args.e2e_jobs

    def job():
        c = B.gempe_create(rp_pin, ci_pin, d, p, stream=stream)
        B.gempe_step(c, epochs)
        B.gempe_positions(c, out_pin)
        used = B.gempe_stats(c)["used"]
        c.close()
        return epochs * m + used

    if e2e_jobs > 0:
        job()   # warm-up (builds nothing new: the library is loaded, the GPU is warm)
        torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_pairs = sum(job() for _ in range(e2e_jobs))
    torch.cuda.synchronize()
    e2e_t = max(time.perf_counter() - t0, 1e-9)
    e2e = {"value": e2e_pairs / e2e_t if e2e_jobs else None, "unit": UNIT,
           "h2d_bytes_per_step": int(rp.nbytes + ci.nbytes),
           "d2h_bytes_per_step": int(out_pin.nbytes),
           "step": f"one {epochs}-epoch embedding job: gempe_create from pinned host CSR, "
                   f"gempe_step({epochs}), gempe_positions to pinned host memory",
           "ms_per_job": 1e3 * e2e_t / e2e_jobs if e2e_jobs else None}
    if world > 1 and e2e_jobs:
        e2e["value"] = sum_ranks(e2e["value"], dev)

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    peak, peak_kind = _peaks()
    block = bool(form.get("block_partners"))
    oriented = d <= 4 and not block and not form.get("sampling")
    units = work_units(rp, k, d, out_degrees=oriented_degrees(rp, ci) if oriented else None)
    bytes_per_sweep = sweep_algorithmic_bytes(n, nnz, d, 0 if block else k, units,
                                              0 if block else accepted / args.steps, oriented=oriented,
                                              row_bytes=position_row_bytes(d, form.get("precision")))
    if block and form.get("precision") and d in (16, 32, 64):
        bytes_per_sweep += tile_algorithmic_bytes(n, d, (n + 127) // 128)
    sweep_s = statistics.mean(sweep_ms) / 1e3
    achieved = bytes_per_sweep / sweep_s / 1e9
    traffic = _profile_traffic(kernel_source_hash(), workload)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": statistics.mean(step_ms), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16 positions, f32 sums" if form.get("precision") else "f32", "data": "synthetic",
        "config": {"workload": workload, "n": n, "m": m, "d": d,
                   "sampling": "block 128x64" if form.get("block_partners") else f"k={k} per vertex",
                   "sigma_every": 1,
                   "step": "one epoch: gempe_step(ctx, 1), a replay of the captured epoch graph",
                   "l2": "flushed between steps (256 MiB write outside the timed events)",
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
        "pairs_per_epoch": pairs / args.steps,
        "sigma_fit_steps_last": s1["sigma_iters"],
        "sweep_ms": statistics.mean(sweep_ms),
        "split_epoch_ms": statistics.mean(split_ms),
        "update_ms": statistics.mean(split_ms) - statistics.mean(sweep_ms),
        "roofline": {"bound": "hbm",
                     "kernel": "k_sweep + k_tile_tc" if (block and form.get("precision")) else "k_sweep",
                     "achieved": achieved, "peak": peak,
                     "peak_kind": f"{peak_kind} HBM copy GB/s", "unit": "GB/s", "frac": achieved / peak,
                     "algorithmic_bytes_per_launch": bytes_per_sweep, "traffic": traffic,
                     "note": "sweep window = events around gempe_sweep in a second pass of as many flushed "
                             "epochs inside the timed region (sweep kernel with the next epoch's sampler "
                             "running beside it)"},
        "sampler_algorithmic_bytes_per_launch": sampler_algorithmic_bytes(n, k, draws / args.steps),
        "exact_pe": exact,
        "clocks": clk,
        "e2e": e2e,
        # per epoch: the sweep (+ the tensor-core tiles), the update, the next epoch's sampler; two passes
        "gpu_launches": (4 if (block and form.get("precision") and d in (16, 32, 64)) else 3) * 2 * args.steps,
        "wall_s_timed_region": wall,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, budget_s=args.cpu_budget)
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def run_batch(args):
    """The batched form: every step is one epoch of all graphs of the batch
    (gempe_batch_step(b, 1): one CUDA-graph launch whose per-dimension
    branches run concurrently)."""
    import numpy as np
    import torch

    from paper_2011_03479_gb300 import binding as B
    from paper_2011_03479_gb300 import inputs

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    workload = args.workload
    w = inputs.sbm_batch_256()
    graphs = w["graphs"]
    k, epochs = w["k"], w["epochs"]
    G = len(graphs)
    form = FORMS[workload]
    p = B.gempe_default_params(neg_per_vertex=k, seed=inputs.EMBED_SEED, **form)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    desc = [(g["row_ptr"], g["col_idx"], g["d"]) for g in graphs]
    m_tot = sum(len(g["col_idx"]) // 2 for g in graphs)
    n_tot = sum(len(g["row_ptr"]) - 1 for g in graphs)

    t_create0 = time.perf_counter()
    b = B.gempe_batch_create(desc, p, stream=stream)
    create_s = time.perf_counter() - t_create0
    shapes = {d: B.gempe_batch_shape(b, d) for d in sorted({g["d"] for g in graphs})}
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush.zero_()
            B.gempe_batch_step(b, 1)
        torch.cuda.synchronize()
        used0 = sum(B.gempe_batch_stats(b, q)["used"] for q in range(G))
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        clocks = ClockSampler(local)
        clocks.start()
        wall0 = time.perf_counter()
        for e0, e1 in ev:
            flush.zero_()
            e0.record(stream)
            B.gempe_batch_step(b, 1)
            e1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
        clk = clocks.stop()
        stats = [B.gempe_batch_stats(b, q) for q in range(G)]
    used = sum(s["used"] for s in stats) - used0
    step_ms = [a.elapsed_time(c) for a, c in ev]
    pairs = args.steps * m_tot + used
    t_total = sum(step_ms) / 1e3
    t_all, pairs_all = combine_ranks(t_total, pairs, dev)
    value = pairs_all / t_all
    b.close()

    # the plain form: every graph in its own FP32 context, one after the other
    alone_steps = min(args.steps, 20) if not args.no_alone_baseline else 0
    alone_pairs, alone_s = 0, 0.0
    pa = B.gempe_default_params(neg_per_vertex=k)
    ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for q, g in enumerate(graphs if alone_steps else []):
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
    alone_value = alone_pairs / alone_s if alone_s else None

    # end to end: one batch job (create from pinned host CSR, `epochs` epochs, positions back)
    pinned = [(torch.from_numpy(g["row_ptr"]).pin_memory().numpy(), torch.from_numpy(g["col_idx"]).pin_memory().numpy(),
               g["d"]) for g in graphs]
    e2e = None
    if args.e2e_jobs > 0:
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
        e2e = {"value": e2e_pairs / e2e_t, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "step": f"one batch job: gempe_batch_create of {G} graphs from pinned host CSR (host validation "
                       f"included), gempe_batch_step({epochs}), gempe_batch_positions of every graph into pinned memory",
               "ms_per_job": 1e3 * e2e_t}
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    peak, peak_kind = _peaks()
    # algorithmic bytes of one epoch's sweeps, all packs (they run concurrently)
    acc_per_epoch = used / args.steps
    byts = 0.0
    for g in graphs:
        rp, ci, d = g["row_ptr"], g["col_idx"], g["d"]
        n = len(rp) - 1
        sh = shapes[d]
        oriented = d <= 4 and sh.get("kernel", 0) == 0
        units = work_units(rp, k, d, edge_chunk=sh["unit"], unit_pairs=sh["unit"],
                           out_degrees=oriented_degrees(rp, ci) if oriented else None, kernel=sh.get("kernel", 0))
        byts += sweep_algorithmic_bytes(n, len(ci), d, k, units, acc_per_epoch * (n / n_tot), oriented=oriented,
                                        row_bytes=position_row_bytes(d, form.get("precision")))
    step_s = statistics.mean(step_ms) / 1e3
    achieved = byts / step_s / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": statistics.mean(step_ms), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16 positions (d >= 8), f32 sums" if form.get("precision") else "f32", "data": "synthetic",
        "config": {"workload": workload, "graphs": G, "n_total": n_tot, "m_total": m_tot,
                   "dims": {str(d): sum(1 for g in graphs if g["d"] == d) for d in shapes}, "k": k,
                   "step": "one epoch of every graph: gempe_batch_step(b, 1), one CUDA-graph launch",
                   "l2": "flushed between steps (256 MiB write outside the timed events)",
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
        "pairs_per_epoch": pairs / args.steps,
        "shapes": {str(d): sh for d, sh in shapes.items()},
        "create_s": create_s,
        "alone_fp32": {"value": alone_value, "unit": UNIT, "ratio": value / alone_value if alone_value else None,
                       "how": f"each graph in its own FP32 context (gempe_create + gempe_step), one after the "
                              f"other, {alone_steps} epochs each, CUDA events around each graph's epochs"},
        "roofline": {"bound": "hbm", "kernel": "epoch (sweeps of all packs, concurrent)", "achieved": achieved,
                     "peak": peak, "peak_kind": f"{peak_kind} HBM copy GB/s", "unit": "GB/s", "frac": achieved / peak,
                     "algorithmic_bytes_per_launch": byts, "traffic": None,
                     "note": "sweep algorithmic bytes of all packs over the whole epoch time"},
        "clocks": clk,
        "e2e": e2e,
        "gpu_launches": args.steps * (3 * len(shapes)),
        "wall_s_timed_region": wall,
    }
    if not args.no_cpu_baseline:
        import oracle
        oracle.build()
        budget, t_used, pairs_cpu, done = args.cpu_budget, 0.0, 0, []
        for q, g in enumerate(graphs):
            if t_used > budget:
                break
            wq = dict(name=f"graph {q}", row_ptr=g["row_ptr"], col_idx=g["col_idx"], d=g["d"], k=k)
            pq, tq, _ = oracle_epochs(wq, 1)
            pairs_cpu += pq
            t_used += tq
            done.append(q)
        line["cpu_baseline"] = {"value": pairs_cpu / t_used, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"one FP64 oracle epoch of each of graphs {done[0]}..{done[-1]} "
                                          f"({len(done)} of {G}), one thread"}
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def run_serve(args):
    """The serving form.  --steps jobs (at most SERVE_MAX_JOBS) arrive as a
    Poisson stream (mean 50 per second): each an R-MAT graph with scale
    uniform in 10..18 and edge factor
    uniform in 8..16 (a pool of two graphs per scale, generated before the
    timed region), d from {2, 32, 128}, 100-300 epochs, k = 10, its own seed.
    They are submitted through gempe_server_submit at their arrival times to a
    server with a 120 GB budget and 32 job slots; the line reports the
    pair-update throughput over the whole run and the p50/p99 completion
    latency (arrival to positions on the host).  --warmup jobs run first,
    untimed."""
    import numpy as np
    import torch

    from paper_2011_03479_gb300 import binding as B
    from paper_2011_03479_gb300 import inputs

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    rng = np.random.default_rng(5000 + rank)
    pool = {}
    for scale in range(10, 19):
        pool[scale] = []
        for r in range(2):
            ef = int(rng.integers(8, 17))
            rp, ci = inputs.rmat(scale, ef, seed=5001 + 100 * scale + r)
            pool[scale].append((rp, ci, ef))
    k = 10
    budget = 120 * (1 << 30)
    p = B.gempe_default_params(neg_per_vertex=k, seed=inputs.EMBED_SEED, **FORMS[args.workload])

    def draw_job(q):
        scale = int(rng.integers(10, 19))
        rp, ci, ef = pool[scale][int(rng.integers(0, 2))]
        return dict(rp=rp, ci=ci, d=int(rng.choice([2, 32, 128])), epochs=int(rng.integers(100, 301)),
                    seed=inputs.EMBED_SEED ^ (q + 1), scale=scale, ef=ef)

    srv = B.gempe_server_create(budget, max_jobs=32, params=p)
    for q in range(args.warmup):
        j = draw_job(-1 - q)
        jid = B.gempe_server_submit(srv, j["rp"], j["ci"], j["d"], 20, j["seed"])
        B.gempe_server_wait(srv, jid, 600000)
        B.gempe_server_result(srv, jid)
    jobs = [draw_job(q) for q in range(min(args.steps, SERVE_MAX_JOBS))]
    gaps = rng.exponential(1.0 / 50.0, size=len(jobs))
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    t0 = time.perf_counter()
    ids = []
    t_next = 0.0
    for j, g in zip(jobs, gaps):
        t_next += g
        dt = t_next - (time.perf_counter() - t0)
        if dt > 0:
            time.sleep(dt)
        ids.append(B.gempe_server_submit(srv, j["rp"], j["ci"], j["d"], j["epochs"], j["seed"]))
    infos = [B.gempe_server_wait(srv, i, 3600 * 1000) for i in ids]
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    for i in ids:
        B.gempe_server_result(srv, i)
    stats = B.gempe_server_stats(srv)
    # capacity: the first jobs again, all submitted at once (closed loop)
    cap_jobs = jobs[: min(len(jobs), 100)]
    cids = [B.gempe_server_submit(srv, j["rp"], j["ci"], j["d"], j["epochs"], j["seed"]) for j in cap_jobs]
    cinfos = [B.gempe_server_wait(srv, i, 3600 * 1000) for i in cids]
    for i in cids:
        B.gempe_server_result(srv, i)
    srv.close()
    cap_span = (max(c["done_ns"] for c in cinfos) - min(c["submit_ns"] for c in cinfos)) / 1e9
    capacity = sum(c["pairs"] for c in cinfos) / cap_span
    sub = np.array([inf["submit_ns"] for inf in infos], dtype=np.float64)
    adm = np.array([inf["admit_ns"] for inf in infos], dtype=np.float64)
    done = np.array([inf["done_ns"] for inf in infos], dtype=np.float64)
    pairs = float(sum(inf["pairs"] for inf in infos))
    span = (done.max() - sub.min()) / 1e9
    lat = (done - sub) / 1e6
    wait = (adm - sub) / 1e6
    arrivals = (sub.max() - sub.min()) / 1e9
    value = sum_ranks(pairs / span, torch.device("cuda", local))
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    h2d = float(np.mean([j["rp"].nbytes + j["ci"].nbytes for j in jobs]))
    d2h = float(np.mean([4 * (len(j["rp"]) - 1) * j["d"] for j in jobs]))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * span / len(jobs), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "jobs": len(jobs), "arrival_rate_per_s": 50,
                   "scale": "U{10..18}", "edge_factor": "U{8..16}", "d": [2, 32, 128], "epochs": "U{100..300}",
                   "k": k, "budget_bytes": budget, "max_jobs": 32,
                   "step": "one job: arrival to positions on the host (gempe_server_submit .. gempe_server_result)",
                   "l2": "inputs (many jobs' device state) larger than L2",
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "mean": float(lat.mean()), "max": float(lat.max())},
        "queue_wait_ms": {"p50": float(np.percentile(wait, 50)), "p99": float(np.percentile(wait, 99))},
        "offered_pairs_per_s": pairs / max(arrivals, 1e-9),
        "capacity_pairs_per_s": capacity,
        "capacity_note": f"{len(cap_jobs)} of the same jobs submitted at once; when the offered load is above "
                         "this the latency is dominated by the queue",
        "peak_device_bytes": stats["peak_bytes_in_use"],
        "failed_jobs": stats["failed"],
        "roofline": None,
        "clocks": clk,
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "step": "one job through the public serving calls (submit from host CSR, result to host)"},
        # per job: set-up (edge set, symmetry check, positions, and for d <= 4 the
        # oriented CSR: count, three scan passes, fill) and per epoch the sweep,
        # the update and the next epoch's sampler
        "gpu_launches": int(sum(3 + (5 if j["d"] <= 4 else 0) + 3 * j["epochs"] for j in jobs)),
        "gpu_launches_note": "counted from the engine's launch structure (set-up and three kernels per epoch per job)",
        "wall_s_timed_region": wall,
    }
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_2011_03479_gb300 import inputs
    oracle.build()
    w = inputs.WORKLOADS[WORKLOAD]()
    m = len(w["col_idx"]) // 2
    _, _, x = oracle_epochs(w, args.warmup) if args.warmup else (0, 0, None)
    times, pairs = [], 0
    for s in range(args.steps):
        p, t, x = oracle_epochs(w, 1, x0=x)
        times.append(t)
        pairs += p
    value = pairs / sum(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": len(w["row_ptr"]) - 1, "m": m, "d": w["d"], "k": w["k"],
                   "step": "one epoch of the FP64 CPU oracle"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} timed epochs of {WORKLOAD} after {args.warmup} warm-up epochs"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["gempe", "reference"], default="gempe")
    ap.add_argument("--e2e-jobs", type=int, default=3)
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-alone-baseline", action="store_true",
                    help="batched workloads: leave out the every-graph-alone comparison (measured after the timed region)")
    ap.add_argument("--workload", choices=sorted(FORMS), default=WORKLOAD,
                    help="graph-drawing workload (default) or the representation-learning forms")
    args = ap.parse_args()
    if args.impl == "reference":
        if args.steps > 50:
            args.steps = 50      # each oracle epoch takes a fraction of a second: keep the run bounded
        run_reference(args)
    elif args.workload in BATCH_WORKLOADS:
        run_batch(args)
    elif args.workload in SERVE_WORKLOADS:
        run_serve(args)
    else:
        run_gempe(args)


if __name__ == "__main__":
    main()
