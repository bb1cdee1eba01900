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
