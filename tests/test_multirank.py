"""Host-side logic of the multi-rank benchmark run, exercised with two gloo
ranks on the CPU: every rank times its own replica, the job's time is the
maximum over ranks, the job's throughput counts every rank's cells over that
time, replicas share no data (each rank's replica ends where the same replica
run alone ends, bit for bit), and only rank 0 reports (the reference arm
exits on the other ranks without work)."""
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


def _replica(seed, steps, world=1):
    """A small seeded replica (oracle, periodic box with a moving marker
    pair), stepped with a barrier between steps as the benchmark's replicas
    are; returns its final populations."""
    import numpy as np
    import oracle
    from paper_2206_01683_b300 import inputs
    shape = (12, 10, 8)
    rho, u = inputs.random_fields(shape, seed=seed, u_amp=0.01, rho_amp=0.005)
    o = oracle.Oracle(shape, 0.7)
    o.init_fields(rho, u)
    rng = np.random.default_rng(seed)
    X0 = rng.uniform(3.0, 6.0, (2, 3))
    U = rng.uniform(-0.01, 0.01, (2, 3))
    for n in range(steps):
        o.set_markers(X0 + U * n, U, np.ones(2))
        o.step()
        if world > 1:
            dist.barrier()
    return o.populations()


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r, w, local = bench.dist_info()
    assert (r, w, local) == (rank, world, rank)
    slowest = bench._max_over_ranks(10.0 + 3.0 * rank, world)
    mlups = bench.job_mlups(world, 1000, 20, slowest)
    pops = _replica(100 + rank, 6, world)
    class A:
        steps, warmup = 2, 3
    ref = bench.run_reference(A) if rank == 1 else "skipped"
    out.put((rank, slowest, ref, mlups, pops))
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
    # both ranks' cells over the slowest rank's time: 2 x 1000 x 20 / 13 ms
    assert res[0][3] == res[1][3] == pytest.approx(2 * 1000 * 20 / 13e-3 / 1e6, rel=1e-12)
    # each replica equals the same replica run alone, and the two differ
    import numpy as np
    for rank in range(2):
        assert np.array_equal(res[rank][4], _replica(100 + rank, 6))
    assert not np.array_equal(res[0][4], res[1][4])
