"""The multi-GPU path of bench.py is replicas only: each rank runs its own
instance, the job time is the max over ranks, and the reference arm runs on
rank 0 alone.  These checks run that host logic as two gloo ranks on the CPU."""

import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, loc = bench.dist_setup()
        t = bench.reduce_max(1.5 + rank, w)          # rank 1 is the slow replica
        q.put((rank, w, r, loc, t))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1]
    for rank, w, r, loc, t in out:
        assert w == 2 and r == rank and loc == rank
        assert t == 2.5                               # max over ranks


def test_reference_arm_is_silent_off_rank_zero(capsys):
    sys.path.insert(0, ROOT)
    import bench

    class A:
        steps, warmup = 1, 1

    bench.run_reference(A(), world=2, rank=1)
    assert capsys.readouterr().out == ""
