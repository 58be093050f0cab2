"""The benchmark's several-GPU logic on CPU: two gloo ranks (no GPU).

Each rank takes its own problem of the same sizes (weak scaling, no data-path
collective); the job's step time is the slowest rank's, reached with one
all-reduce, and the job's throughput counts every rank's units.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402
from paper_1508_04245_gb300 import workloads as W  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms_local = [12.5, 17.25][rank]
        ms = bench.max_over_ranks(ms_local, world, "cpu")
        wl = bench.rank_workload(W.WORKLOADS["square16_k2"], rank)
        verts, elems = wl.mesh()
        out.put((rank, ms, bench.job_throughput(1000.0, world, ms), wl.seed, float(verts.sum()),
                 int(elems.sum())))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank_and_own_problems():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, ms0, v0, s0, x0, e0), (r1, ms1, v1, s1, x1, e1) = res
    assert ms0 == ms1 == 17.25                       # max over ranks, seen by every rank
    assert v0 == v1 == pytest.approx(2 * 1000.0 / 17.25e-3)
    assert s0 == W.WORKLOADS["square16_k2"].seed and s1 != s0
    assert e0 == e1                                  # same sizes and connectivity


def test_rank_workloads_differ_where_the_seed_enters():
    wl = W.WORKLOADS["square256_k4"]
    a, b = bench.rank_workload(wl, 0), bench.rank_workload(wl, 1)
    assert a is wl and b.n_elem == a.n_elem and b.k == a.k
    va, _ = W.square_mesh(8, a.jitter, a.seed)
    vb, _ = W.square_mesh(8, b.jitter, b.seed)
    assert not np.allclose(va, vb)
    assert bench.max_over_ranks(3.0, 1, "cpu") == 3.0
