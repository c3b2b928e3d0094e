"""The N > 1 bench path on CPU: two replicas (gloo, world size 2) agree on the
slowest replica's time and on the whole-job rate; the reference arm runs on
rank 0 only (the other rank returns at once)."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _replica(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import bench

    dist, r, ws = bench._dist()
    assert dist.get_backend() == "gloo" and r == rank and ws == world
    slowest = bench.max_over_ranks(dist, 10.0 + 5.0 * rank)  # rank 1 is the slow replica
    rate = bench.whole_job_rate(4, ws, slowest)

    class Args:
        steps, warmup = 1, 3

    ref_rc = bench.run_reference(Args) if rank == 1 else 0  # rank != 0 does no work
    out.put((rank, slowest, rate, ref_rc))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_agree_on_slowest_time_and_rate():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_replica, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, rate, ref_rc in res:
        assert slowest == 15.0
        assert rate == pytest.approx(4 * 2 / 15.0)
        assert ref_rc == 0
