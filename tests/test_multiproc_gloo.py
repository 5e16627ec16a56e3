"""World-size-2 checks of the multi-rank bookkeeping on CPU (gloo).

The path does not shard a single system: N GPUs run N independent replicas
(one system per rank, no collective on the data path).  What the ranks do
share is the benchmark's job accounting: the slowest rank's time and the sum
of all ranks' bytes.  These tests run that accounting, and a per-rank oracle
solve of a rank-seeded system, as two gloo processes on the host.
"""

import os
import socket

import pytest
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
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, b = bench.job_totals(10.0 + 5.0 * rank, 1000 * (rank + 1), world, torch.device("cpu"))
    # every replica solves its own system; the accounting sums their bytes
    import numpy as np
    import oracle
    import workloads as W
    A = W.fd_helmholtz_box(6, kh=0.3 + 0.2 * rank, damping=0.05)
    rhs = W.complex_normal(np.random.default_rng(4000 + rank), A.n)
    x, info = oracle.bicgstab(A, rhs, tol=1e-10, maxit=500)
    _, nb = bench.job_totals(0.0, bench.solve_bytes(A.n, A.nnz, info.iters), world, torch.device("cpu"))
    dist.barrier()
    q.put((rank, t, b, info.status, info.iters, nb, bench.solve_bytes(A.n, A.nnz, info.iters)))
    dist.destroy_process_group()


def test_job_totals_two_ranks():
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    for rank, t, b, status, iters, nb, mine in res:
        assert t == 15.0            # slowest rank
        assert b == 3000            # all ranks' bytes
        assert status == 0 and iters > 0
    assert res[0][5] == res[1][5] == res[0][6] + res[1][6]


def test_single_rank_is_identity():
    import bench
    assert bench.job_totals(3.0, 7, 1, None) == (3.0, 7)
