"""The N > 1 path of bench.py (independent replicas, barrier, max over ranks) with two gloo
ranks on the CPU."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    import torch.distributed as dist
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ws, r, local = bench.dist_env()
    ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
    dist.barrier()
    ms_max = bench.max_over_ranks(ms)
    mlups = bench.whole_job_mlups(1000, 20, ws, ms_max)
    out.put((rank, ws, r, local, ms_max, mlups))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    mp = pytest.importorskip("torch.multiprocessing")
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
    for rank, ws, r, local, ms_max, mlups in res:
        assert ws == 2 and r == rank and local == rank
        assert ms_max == 15.0
        assert mlups == pytest.approx(2 * 1000 * 20 / 15e-3 / 1e6)


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.whole_job_mlups(100, 10, 1, 2.0) == pytest.approx(100 * 10 / 2e-3 / 1e6)
