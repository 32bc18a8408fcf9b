"""The benchmark's multi-rank path on CPU (gloo, world size 2): each rank
runs its own node set, the step time is the maximum over ranks and the value
counts the units of all ranks (weak scaling, no data-path collective)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    rk = bench.Ranks("gloo")
    # a per-rank seed gives each rank its own node set
    import nodesets as NS
    ns = NS.disk_holes(2000, seed=rk.rank)
    ms_local = 10.0 + 5.0 * rk.rank          # rank 1 is the slow one
    (ms_max,) = rk.max([ms_local])
    (n_all,) = rk.sum([ns.N])
    value = bench.throughput(n_all, ms_max, steps=4)
    rk.barrier()
    q.put((rk.rank, ns.N, float(ns.pts[0, 0]), ms_max, value))
    rk.close()


@pytest.mark.timeout(120)
def test_two_ranks_reduce_max_time_and_sum_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=100) for _ in procs)
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    (r0, n0, x0, m0, v0), (r1, n1, x1, m1, v1) = out
    assert m0 == m1 == 15.0                       # max over ranks
    assert v0 == v1 == pytest.approx((n0 + n1) * 4 / 15e-3)
    assert x0 != x1                               # different node sets per rank
