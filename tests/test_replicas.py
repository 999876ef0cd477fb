"""The multi-GPU form is replicas only (each rank solves its own copy; no
collective on the data path).  The ranks meet once, after the timed region:
the job's time is the slowest rank's, and throughput counts every rank's
units.  Checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as tmp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    t = bench.max_over_ranks(10.0 + 5.0 * rank, world, device="cpu")
    q.put((rank, t, bench.job_rate(10, world, t)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [15.0, 15.0]
    assert res[0][2] == pytest.approx(2 * 10 / 0.015)


def test_single_rank_is_identity():
    import bench

    assert bench.max_over_ranks(7.5, 1) == 7.5
    assert bench.job_rate(10, 1, 100.0) == pytest.approx(100.0)
