"""Host-side logic of the multi-rank benchmark run, exercised with two gloo
ranks on the CPU: every rank times its own replica, the job's time is the
maximum over ranks, and only rank 0 reports (the reference arm exits on the
other ranks without work)."""
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


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r, w, local = bench.dist_info()
    assert (r, w, local) == (rank, world, rank)
    slowest = bench._max_over_ranks(10.0 + 3.0 * rank, world)
    class A:
        steps, warmup = 2, 3
    ref = bench.run_reference(A) if rank == 1 else "skipped"
    out.put((rank, slowest, ref))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank_and_only_rank0_reports():
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
    assert res[0][1] == res[1][1] == 13.0
    assert res[1][2] is None          # the reference arm does no work off rank 0
