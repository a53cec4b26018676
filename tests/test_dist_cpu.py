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


def test_reference_arm_json_line():
    """bench.py --impl reference on one rank: the oracle timed on the host,
    printed as one JSON line with the contract's keys (the ratio's divisor)."""
    import json
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("{")][-1]
    d = json.loads(line)
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 0
    assert d["unit"] == "Mcells/s" and d["higher_is_better"] is True and d["value"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"] and d["metric"]
