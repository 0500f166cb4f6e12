"""The multi-GPU host logic of bench.py on CPU ranks (gloo, world size 2).

Every run in this project has one GPU, so the N > 1 paths are checked here:
the job time is the slowest rank's (max over ranks), and the batched
workload gives every rank its own independent batch (sharding by system,
no collective on the data path)."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench
    from paper_2011_01850_gb300 import inputs as I
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    try:
        got = bench.max_over_ranks(1.5 + rank, world, device="cpu")
        sysr = I.batched_convdiff2d(count=4, nmin=50, nmax=400, seed=bench.batched_seed(rank))
        sig = float(sum(np.sum(A[2]) + np.sum(b) for A, b in sysr))
        sigs = [None] * world
        dist.all_gather_object(sigs, sig)
        q.put((rank, got, sigs))
    finally:
        dist.destroy_process_group()


def test_two_cpu_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, sigs in out:
        assert got == 2.5  # the slower rank's time, on every rank
        assert sigs[0] != sigs[1]  # independent batches per rank


def test_one_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, 1) == 3.25
    assert bench.batched_seed(0) == bench.SEED
