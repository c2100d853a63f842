"""Weak scaling over ranks (bench.py under torchrun), tested on the CPU with
two gloo ranks: rank r integrates prisms r E .. (r+1) E - 1 of a 2E-prism
mesh, generated for its slice only; the gathered shards are exactly the
whole mesh and its coefficients (the elements are independent, so no data
moves between ranks), and the reported time is the largest over the ranks."""
import socket

import numpy as np

from _multirank import worker
from paper_1310_1191_gb300 import inputs


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_rank_shards_and_max_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    E, world, port = 750, 2, _free_port()
    procs = [ctx.Process(target=worker, args=(r, world, port, E, q)) for r in range(world)]
    for p in procs:
        p.start()
    try:
        X, C, t = q.get(timeout=180)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.terminate()
    assert all(p.exitcode == 0 for p in procs)
    assert np.array_equal(X, inputs.prism_mesh(world * E))
    assert np.array_equal(C, inputs.coefficients(world * E))
    assert t == 13.0


def test_shard_of_one_rank_is_the_plain_mesh():
    import bench
    X, C = bench.shard_inputs(500, 0, 1)
    assert np.array_equal(X, inputs.prism_mesh(500)) and np.array_equal(C, inputs.coefficients(500))
    # a middle shard of a three-rank mesh equals the slice of the whole mesh
    X1, C1 = bench.shard_inputs(400, 1, 3)
    assert np.array_equal(X1, inputs.prism_mesh(1200)[400:800])
    assert np.array_equal(C1, inputs.coefficients(1200)[:, 400:800])
