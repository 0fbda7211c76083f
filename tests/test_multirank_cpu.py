"""Multi-rank logic on CPU (gloo, world size 2).

1. The paper's decomposition (Sect. 3, the evaluation is split over n processes
   holding N/n j-particles each, then summed over processes): each rank
   evaluates all listed i-particles against its half of the j-particles with
   the oracle (the other half given zero mass), an all-reduce sums the partial
   acc/jerk/snap, and the sum equals the single-process evaluation.
2. The benchmark's whole-job aggregation over ranks: maximum time, summed
   interactions.
"""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import oracle
    import bench
    from paper_1207_2367_gb300 import inputs

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n = 300
        p = inputs.plummer(n, 17, imf="salpeter")
        ap = np.random.default_rng(3).normal(size=(n, 3))
        idx = np.arange(0, n, 7, dtype=np.int32)
        mine = np.zeros(n, dtype=bool)
        mine[rank * n // world:(rank + 1) * n // world] = True
        mass = np.where(mine, p.mass, 0.0)        # this rank's j-particles only
        parts = oracle.evaluate(mass, p.pos, p.vel, ap, 1e-3, idx)
        t = torch.tensor(np.concatenate([x.ravel() for x in parts]))
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        full = np.concatenate([x.ravel() for x in oracle.evaluate(p.mass, p.pos, p.vel, ap, 1e-3, idx)])
        err = float(np.abs(t.numpy() - full).max() / np.abs(full).max())
        ms, inter = bench.aggregate(10.0 + rank, 1000 * (rank + 1), dist, "cpu")
        q.put((rank, err, ms, inter))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_j_partition_and_rank_aggregation_with_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    out = [q.get(timeout=240) for _ in range(world)]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    for rank, err, ms, inter in out:
        assert err < 1e-13
        assert ms == 11.0            # the slower rank
        assert inter == 3000         # 1000 + 2000
