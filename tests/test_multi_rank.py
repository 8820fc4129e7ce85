"""Host-side logic of the multi-GPU benchmark path on CPU: two gloo ranks
exchange their timings the way `bench.py` does (barrier, max over ranks,
aggregate over all replicas) and draw different resonator variants."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    ws, r, local = bench.dist_env()
    assert (ws, r, local) == (world, rank, rank)
    d = bench.init_dist(ws, "gloo")
    bench.barrier(d)
    ms = 10.0 + 5.0 * rank                     # rank 1 is the slower one
    ms_max = bench.max_over_ranks(d, ms)
    total = bench.sum_over_ranks(d, 1.0)
    value = bench.aggregate(1000, 100, ms_max, ws)
    from paper_2305_13419_gb300 import workloads as W
    w = W.cpw_small(seed=bench.replica_seed(rank))
    out.put((rank, ms_max, total, value, float(w.sigma.sum())))
    d.barrier()
    d.destroy_process_group()


def test_two_gloo_ranks_reduce_like_the_benchmark():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, m0, t0, v0, s0), (r1, m1, t1, v1, s1) = res
    assert m0 == m1 == 15.0          # both ranks see the slowest rank's time
    assert t0 == t1 == 2.0
    assert v0 == v1 == pytest.approx(2 * 1000 * 100 / 15e-3 / 1e9)
    assert s0 != s1                  # each replica is its own resonator variant
