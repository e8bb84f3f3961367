"""The multi-rank host logic on CPU ranks (gloo, world size 2).

- Eq. 8 of the paper: the transform of all points is the sum of the
  transforms of the rank-local subsets (spatial halves of the box, as the
  paper's Split(box) makes subcells); an all-reduce of the per-rank oracle
  adjoints equals the whole.
- The benchmark's aggregation: every rank runs its own problems, the step time
  is the maximum over ranks and the throughput counts all ranks' points.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, results):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import ndft
        from paper_2001_01583_gb300 import inputs
        N = (8, 6, 10)
        x = inputs.uniform_points(400, 3, seed=3)
        f = inputs.complex_normal(400, seed=4)
        mine = (x[:, 0] >= 0.0) if rank == 0 else (x[:, 0] < 0.0)   # split the box in two subcells
        part = ndft.adjoint(x[mine], f[mine], N, threads=1)
        t = torch.from_numpy(np.ascontiguousarray(part.view(np.float64)))
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        # the benchmark's timing reduction: max over ranks
        ms = torch.tensor([1.5 + rank], dtype=torch.float64)
        dist.all_reduce(ms, op=dist.ReduceOp.MAX)
        if rank == 0:
            whole = ndft.adjoint(x, f, N, threads=1)
            summed = t.numpy().view(np.complex128).reshape(N)
            results.put((float(np.max(np.abs(summed - whole)) / np.max(np.abs(whole))), float(ms.item())))
    finally:
        dist.destroy_process_group()


def test_subcell_split_all_reduce_equals_whole():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    err, ms = q.get(timeout=10)
    assert err < 1e-12
    assert ms == 2.5
