"""Multi-process plumbing of bench.py on CPU ranks (gloo, world size 2).

The solve does not exchange data between GPUs: N ranks run N replicas
(weak scaling) and only the barrier and the max-over-ranks timing cross
ranks.  These tests run that plumbing, and the reference arm's rank
handling, as two gloo processes on the host.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as td  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "WORLD_SIZE": str(world),
                       "RANK": str(rank), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import bench
    d = bench.Dist()
    try:
        assert d.world == world and d.rank == rank and d.pg is not None
        d.barrier()
        # max over ranks of a per-rank time, as the timed region reports it
        m = d.max(10.0 + rank)
        # the reference arm: rank 0 alone runs; others return None and exit 0
        class A:
            workload = "const32"
            kappa = None
            steps = 0
            warmup = 0
        ref = bench.run_reference(A(), d) if rank != 0 else "skipped"
        q.put((rank, m, ref))
    finally:
        d.close()


def test_two_rank_barrier_max_and_reference_rank_handling():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=5) for _ in range(2))
    assert [o[1] for o in out] == [11.0, 11.0]   # both ranks see the max
    assert out[1][2] is None                      # rank 1 does no reference work
