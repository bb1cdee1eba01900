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
