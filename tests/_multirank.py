"""Worker of the two-rank CPU test (gloo): one process per rank runs the
multi-rank host logic of bench.py."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def worker(rank, world, port, E, q):
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import numpy as np
    import torch
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        X, C = bench.shard_inputs(E, rank, world)
        Xt, Ct = torch.from_numpy(np.ascontiguousarray(X)), torch.from_numpy(np.ascontiguousarray(C))
        xs = [torch.empty_like(Xt) for _ in range(world)]
        cs = [torch.empty_like(Ct) for _ in range(world)]
        dist.all_gather(xs, Xt)
        dist.all_gather(cs, Ct)
        # each rank reports a different step time; the bench keeps the largest
        t = bench.max_over_ranks(10.0 + 3.0 * rank, world)
        if rank == 0:
            q.put((np.concatenate([x.numpy() for x in xs]), np.concatenate([c.numpy() for c in cs], axis=1), t))
        dist.barrier()
    finally:
        dist.destroy_process_group()
