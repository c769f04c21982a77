"""The N > 1 host path of the benchmark on CPU (gloo, world size 2): each rank
runs an independent replica, the job time is the slowest rank's, and the job
value counts every replica's zone-updates."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.aggregate_ms(10.0 + rank, dist, "cpu")
    q.put((rank, ms, bench.job_value(1000, world, ms)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_time_is_max_over_ranks():
    import torch.multiprocessing as mp

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
    assert [o[1] for o in out] == [11.0, 11.0]
    assert out[0][2] == pytest.approx(1000 * 2 * 2 / 11e-3)


def test_single_rank_needs_no_group():
    import bench
    assert bench.aggregate_ms(7.5, None, "cpu") == 7.5
