"""The multi-GPU reduction of bench.py (replicas: max-over-ranks time, whole-job
rate) run as two gloo ranks on the CPU, rendezvous on 127.0.0.1."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r took 1 + r s for the mixed leg, 3 - r s for the FP64 leg, 0.5 s end to end
    got = bench.max_over_ranks([1.0 + rank, 3.0 - rank, 0.5], world)
    q.put((rank, got, bench.job_rate(world, 65536 * 5, got[0])))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_two_gloo_ranks():
    import torch.multiprocessing as mp
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=180) for _ in range(world)]
    for p in procs:
        p.join(timeout=180)
        assert p.exitcode == 0
    assert sorted(r for r, _, _ in res) == [0, 1]
    for _, got, rate in res:
        assert got == [2.0, 3.0, 0.5]  # every rank holds the maximum of each leg
        assert rate == pytest.approx(2 * 65536 * 5 / 2.0 / 1e6)  # both ranks' dofs / max time


def test_single_rank_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([1.5, 2.5], 1) == [1.5, 2.5]
    assert bench.job_rate(1, 1e6, 2.0) == pytest.approx(0.5)
