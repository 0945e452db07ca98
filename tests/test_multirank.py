"""Multi-process path of bench.py on CPU (gloo, world size 2): each rank owns
an independent disc, the job time is the maximum over ranks and the rate
counts every rank's cells."""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [3.0, 5.0][rank]                     # rank 1 is the slow one
    t = bench.reduce_max(local_ms, world)
    bench.barrier(world)
    rate = bench.whole_job_rate(1000, world, t, 10)

    class A:
        nr, nphi, bifluid = 16, 32, False

    d = bench.workload(A, rank)
    q.put((rank, t, rate, float(d.sigma_g.sum())))
    dist.destroy_process_group()


def test_two_rank_aggregation_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, t0, r0, s0), (_, t1, r1, s1) = res
    assert t0 == t1 == 5.0                          # max over ranks
    assert np.isclose(r0, 2 * 1000 / (0.5e-3))      # both ranks' cells / slowest per-step time
    assert r0 == r1
    assert s0 != s1                                 # independent discs per rank
