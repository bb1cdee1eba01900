"""Worker of the world-size-2 gloo tests (spawned processes import it by name)."""
import os
import sys


def combine(rank, world, port, queue):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        t, p = bench.combine_ranks(1.0 + rank, 100 * (rank + 1))
        v = bench.sum_ranks(2.0 * (rank + 1))
        none = bench.sum_ranks(None)
        queue.put((rank, t, p, v, none))
    finally:
        dist.destroy_process_group()


def shares(rank, world, port, queue):
    """Each rank computes its own share of a 256-graph batch and of a job
    stream; the shares are gathered over gloo."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        sizes = [(q * 7919) % 1000 + 1 for q in range(256)]
        mine = bench.shard_jobs(sizes, world, rank)
        jobs = bench.stream_share(200, world, rank)
        got = [None] * world
        dist.all_gather_object(got, (mine, jobs))
        queue.put((rank, got, sizes))
    finally:
        dist.destroy_process_group()


class OracleShard:
    """A shard engine on the host for the exchange tests: the oracle's terms
    of the anchors [lo, hi) (orc_epoch_range) as the partial sums, and the
    update x_i := y_i / z_i of the own rows with sigma refitted on the summed
    histograms (Fig. 4, Sec. III.F)."""

    def __init__(self, oracle, rp, ci, x0, seed, k, lo, hi, form):
        self.o, self.rp, self.ci, self.seed, self.k = oracle, rp, ci, seed, k
        self.lo, self.hi, self.form = lo, hi, form
        self.x = x0.copy()
        self.sigma, self.epoch = 1.0, 0

    def sweep(self):
        import torch
        r = self.o.epoch(self.rp, self.ci, self.x, self.sigma, self.epoch, self.seed, self.k,
                         anchors=(self.lo, self.hi), **self.form)
        self.parts = [torch.from_numpy(r[f].copy()) for f in ("y", "z", "hist_e", "hist_n")]

    def partials(self):
        return self.parts

    def set_partials(self, tensors):
        self.parts = tensors

    def update(self):
        y, z, he, hn = (t.numpy() for t in self.parts)
        xn = self.x.copy()
        for i in range(self.lo, self.hi):
            if z[i] >= 1e-30:
                xn[i] = y[i] / z[i]
        self.x = xn
        self.sigma = self.o.sigma_fit(he, hn)
        self.epoch += 1

    def positions(self):
        import torch
        return torch.from_numpy(self.x.copy())

    def set_positions(self, x):
        self.x = x.numpy().copy()


def shard_epochs(rank, world, port, queue, form_name):
    """Each rank runs two epochs of its vertex range with the product's
    exchange (ShardRank over gloo) on an oracle-backed engine."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_2011_03479_gb300 import inputs, shard
        oracle.build()
        w = inputs.sbm_1000()
        rp, ci = w["row_ptr"], w["col_idx"]
        forms = {"per-vertex": (2, 5, {}), "block": (16, 0, {"block_partners": 64})}
        d, k, form = forms[form_name]
        ranges = shard.vertex_ranges(rp, world, block=bool(form))
        lo, hi = ranges[rank]
        x0 = oracle.init_positions(len(rp) - 1, d, 99).astype("float64")
        eng = OracleShard(oracle, rp, ci, x0, 99, k, lo, hi, form)
        shard.ShardRank(eng).step(2)
        queue.put((rank, ranges, eng.x, eng.sigma))
    finally:
        dist.destroy_process_group()


class InjectedFailure(RuntimeError):
    """The host-side failure a test plants in one rank's engine."""


class FailingShard(OracleShard):
    """An OracleShard whose sweep raises at epoch `fail_at` (a rank that
    fails between two of the exchange's collectives)."""

    def __init__(self, *args, fail_at, **kw):
        super().__init__(*args, **kw)
        self.fail_at = fail_at

    def sweep(self):
        if self.epoch == self.fail_at:
            raise InjectedFailure(f"injected failure at epoch {self.epoch}")
        super().sweep()


def shard_peer_fails(rank, world, port, queue, timeout_s):
    """Two ranks run the sharded exchange; rank 1's engine fails at its
    second epoch and the rank leaves.  Each rank reports how its step ended:
    rank 1 with the injected failure, rank 0 with the error its next
    collective raises (a closed connection, or the process group's timeout)."""
    import datetime
    import time
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=timeout_s))
    outcome = None
    t0 = time.monotonic()
    try:
        import oracle
        from paper_2011_03479_gb300 import inputs, shard
        oracle.build()
        w = inputs.sbm_1000()
        rp, ci = w["row_ptr"], w["col_idx"]
        lo, hi = shard.vertex_ranges(rp, world)[rank]
        x0 = oracle.init_positions(len(rp) - 1, 2, 99).astype("float64")
        eng = FailingShard(oracle, rp, ci, x0, 99, 5, lo, hi, {}, fail_at=1 if rank == 1 else -1)
        try:
            shard.ShardRank(eng).step(3)
            outcome = ("completed", eng.epoch)
        except InjectedFailure as e:
            outcome = ("injected", eng.epoch, str(e))
        except Exception as e:   # the collective that lost its peer
            outcome = ("collective error", eng.epoch, type(e).__name__)
    finally:
        queue.put((rank, outcome, time.monotonic() - t0))
        if outcome and outcome[0] != "collective error":
            dist.destroy_process_group()
