"""The z-slab partition of the operator on CPU ranks (gloo), against the
single-domain oracle.

The solve shards along z like the paper's domain decomposition (Sec. 4): a
rank owns a contiguous range of planes, needs one plane of each neighbour
(a halo) before a 7-point pass, and contributes partial sums to each inner
product.  These tests run that plan with the oracle's cell-by-cell operator on
2 and 3 gloo processes: halo planes go point to point between neighbouring
ranks, the plates stay with the first and last rank, and inner products are
all-reduced.  The distributed operator equals the single-domain one bit for
bit; the all-reduced inner product equals the single-domain one to rounding.
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as td  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SHAPE = (11, 6, 8)  # (nz, ny, nx): z does not divide evenly among 2 or 3 ranks


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _slab(rank, world, nz):
    base, extra = divmod(nz, world)
    k0 = rank * base + min(rank, extra)
    return k0, k0 + base + (1 if rank < extra else 0)


def _worker(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    from oracle import gmg_oracle as O
    from streamer_inputs import random_coefficient, random_field
    td.init_process_group("gloo", rank=rank, world_size=world)
    try:
        nz, ny, nx = SHAPE
        grid = O.Grid(nx, ny, nz, 1.0, 0.9, 1.3)
        a = random_coefficient(600, SHAPE, 1e3)  # every rank can regenerate the seeded inputs
        x = random_field(601, SHAPE)
        k0, k1 = _slab(rank, world, nz)
        # the rank holds its planes and, after the exchange, one halo plane from each neighbour
        loc_x = np.zeros(SHAPE)
        loc_a = np.zeros(SHAPE)
        loc_x[k0:k1], loc_a[k0:k1] = x[k0:k1], a[k0:k1]
        reqs = []
        recv = {}
        for nb, mine, theirs in ((rank - 1, k0, k0 - 1), (rank + 1, k1 - 1, k1)):
            if 0 <= nb < world:
                send = torch.from_numpy(np.ascontiguousarray(np.stack([x[mine], a[mine]])))
                recv[theirs] = torch.empty((2, ny, nx), dtype=torch.float64)
                reqs.append(td.isend(send, nb))
                reqs.append(td.irecv(recv[theirs], nb))
        for r in reqs:
            r.wait()
        for k, t in recv.items():
            loc_x[k], loc_a[k] = t[0].numpy(), t[1].numpy()
        cells = [(k, j, i) for k in range(k0, k1) for j in range(ny) for i in range(nx)]
        y = O.apply_operator_at(grid, loc_a, loc_x, cells)
        # inner product (x, A x) over the slab, all-reduced
        part = torch.tensor([float(np.dot(x[k0:k1].ravel(), y))], dtype=torch.float64)
        td.all_reduce(part)
        q.put((rank, k0, k1, y, part.item()))
    finally:
        td.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_z_slab_operator_and_inner_product(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sys.path.insert(0, ROOT)
    from oracle import gmg_oracle as O
    from streamer_inputs import random_coefficient, random_field
    nz, ny, nx = SHAPE
    grid = O.Grid(nx, ny, nz, 1.0, 0.9, 1.3)
    a = random_coefficient(600, SHAPE, 1e3)
    x = random_field(601, SHAPE)
    cells = [(k, j, i) for k in range(nz) for j in range(ny) for i in range(nx)]
    ref = O.apply_operator_at(grid, a, x, cells)
    got = np.concatenate([y for _, _, _, y, _ in out])
    assert [(k0, k1) for _, k0, k1, _, _ in out] == [_slab(r, world, nz) for r in range(world)]
    assert np.array_equal(got, ref)  # bit for bit: the same operations per cell
    dot = float(np.dot(x.ravel(), ref))
    for *_, d in out:
        assert d == pytest.approx(dot, rel=1e-14)
    # the single-domain whole-array operator agrees to rounding
    np.testing.assert_allclose(ref, O.apply_operator(grid, a, x).ravel(), rtol=1e-13,
                               atol=1e-13 * np.abs(ref).max())
