"""One graph over several GPUs: vertex-range shards and their exchange.

Sec. III.E parallelises an epoch by splitting the work over threads and
adding up the numerators and denominators of Eq. 3 (y_i, z_i) at the end.
With one GPU per rank the same split is a 1-D partition of the vertices:
rank r evaluates the anchors of its range (their edges, their sampled
non-edges, their tiles) and adds every term into its own copy of all
vertices' sums.  One epoch is then

    sweep (each rank, its anchors)
    sum the sums and the distance histograms over the ranks   (all-reduce)
    update (each rank: its own rows; sigma refitted on the summed histograms,
            so every rank fits the same sigma)
    gather the positions: each rank's own rows to every rank  (all-reduce of
            the rows, the other ranks' rows at zero)

A graph is placed by `vertex_ranges` (consecutive ranges of nearly equal
work, on tiles of 128 vertices in the block form).  `ShardRank` runs the
epochs of one rank with torch.distributed collectives (NCCL between GPUs,
gloo on the host); `local_epochs` runs several shards in one process in
lock step (every exchange a plain sum), which checks the engine's shard mode
on one GPU.  An engine is any object with sweep(), partials() -> tensors,
set_partials(tensors), update(), positions() -> tensor [n, d],
set_positions(tensor) and own rows (lo, hi); `GpuShard` is the engine of
the C ABI (gempe_create_shard), whose work and the exchange's torch
operations run on one stream (a non-default one: ShardRank and
local_epochs make it current around their torch operations).
"""
from __future__ import annotations

import numpy as np

from . import binding as B

BLOCK_T = 128


def vertex_ranges(row_ptr, world: int, block: bool = False) -> list[tuple[int, int]]:
    """`world` consecutive vertex ranges covering [0, n) whose work (CSR
    slots plus one per vertex) differs little; in the block form every cut
    lies on a tile of 128 vertices.  A rank may get an empty range only when
    there are fewer tiles (or vertices) than ranks."""
    rp = np.asarray(row_ptr, dtype=np.int64)
    n = len(rp) - 1
    unit = BLOCK_T if block else 1
    cuts_allowed = np.arange(0, n + 1, unit)
    if cuts_allowed[-1] != n:
        cuts_allowed = np.append(cuts_allowed, n)
    work = rp[cuts_allowed] + cuts_allowed      # work of [0, cut)
    total = work[-1]
    cuts = [0]
    for r in range(1, world):
        target = total * r / world
        q = int(np.searchsorted(work, target))
        q = min(max(q, 0), len(cuts_allowed) - 1)
        if q > 0 and abs(work[q - 1] - target) <= abs(work[q] - target):
            q -= 1
        cuts.append(max(int(cuts_allowed[q]), cuts[-1]))
    cuts.append(n)
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


class GpuShard:
    """The engine of one rank: a shard context (gempe_create_shard) and
    device buffers for the arrays the exchange moves."""

    def __init__(self, row_ptr, col_idx, d: int, lo: int, hi: int, params=None, stream=None, device=None):
        import torch
        self.lo, self.hi = int(lo), int(hi)
        # the context's work and the exchange's torch operations share one
        # stream, which orders them: a given one, else a new one (never the
        # default stream, whose null handle would give the context a stream
        # of its own)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        if self.stream.cuda_stream == 0:
            raise ValueError("a shard needs a non-default stream")
        self.ctx = B.gempe_create_shard(row_ptr, col_idx, d, lo, hi, params, stream=self.stream)
        lay = B.gempe_shard_layout(self.ctx)
        dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        bins = lay["bins"]
        self.n, self.d = len(row_ptr) - 1, d
        self.bufs = [torch.zeros(lay["sum_floats"], dtype=torch.float32, device=dev),   # y - z x and z per row
                     torch.zeros(bins, dtype=torch.int32, device=dev),                 # edge counts
                     torch.zeros(bins, dtype=torch.int32, device=dev),                 # sample counts
                     torch.zeros(bins, dtype=torch.int64, device=dev),                 # anchor-degree sums
                     torch.zeros(bins, dtype=torch.float32, device=dev)]               # weight corrections
        self.x = torch.zeros((self.n, d), dtype=torch.float32, device=dev)

    def sweep(self):
        B.gempe_sweep(self.ctx)

    def partials(self):
        for what, buf in enumerate(self.bufs):
            B.gempe_shard_copy(self.ctx, what, 0, buf)
        return self.bufs

    def set_partials(self, tensors):
        for what, buf in enumerate(tensors):
            B.gempe_shard_copy(self.ctx, what, 1, buf)

    def update(self):
        B.gempe_update(self.ctx)

    def positions(self):
        B.gempe_shard_copy(self.ctx, B.SHARD_POSITIONS, 0, self.x)
        return self.x

    def set_positions(self, x):
        B.gempe_shard_copy(self.ctx, B.SHARD_POSITIONS, 1, x)

    def close(self):
        self.ctx.close()


def _own_rows_only(x, lo, hi):
    """x with the rows outside [lo, hi) set to zero (adding the ranks' copies
    then gathers every rank's own rows exactly)."""
    y = x.clone()
    y[:lo] = 0
    y[hi:] = 0
    return y


def _on_stream(engine):
    """The torch stream context of an engine's stream (none for host engines)."""
    import contextlib
    s = getattr(engine, "stream", None)
    if s is None:
        return contextlib.nullcontext()
    import torch
    return torch.cuda.stream(s)


class ShardRank:
    """The epochs of one rank over a torch.distributed process group."""

    def __init__(self, engine, group=None):
        self.engine = engine
        self.group = group

    def step(self, epochs: int = 1):
        import torch.distributed as dist
        e = self.engine
        with _on_stream(e):
            for _ in range(epochs):
                e.sweep()
                parts = e.partials()
                for t in parts:
                    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=self.group)
                e.set_partials(parts)
                e.update()
                x = _own_rows_only(e.positions(), e.lo, e.hi)
                dist.all_reduce(x, op=dist.ReduceOp.SUM, group=self.group)
                e.set_positions(x)


def local_epochs(engines, epochs: int = 1):
    """Several shards of one graph in one process, in lock step: the same
    exchange as ShardRank with every all-reduce a plain sum.  The engines
    share one stream (GpuShard(..., stream=s) with the same s)."""
    streams = {id(getattr(e, "stream", None)) for e in engines}
    if len(streams) != 1:
        raise ValueError("the shards of local_epochs share one stream")
    with _on_stream(engines[0]):
        for _ in range(epochs):
            for e in engines:
                e.sweep()
            parts = [[t.clone() for t in e.partials()] for e in engines]
            total = [sum(p[q] for p in parts) for q in range(len(parts[0]))]
            for e in engines:
                e.set_partials([t.clone() for t in total])
            for e in engines:
                e.update()
            x = sum(_own_rows_only(e.positions(), e.lo, e.hi) for e in engines)
            for e in engines:
                e.set_positions(x.clone())
