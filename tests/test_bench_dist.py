"""Host-side logic of the multi-rank benchmark (one replica of the workload per
rank, the job's time is the slowest rank's), exercised with two gloo ranks on
the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    total_ms = 1000.0 * (rank + 1)  # rank 1 is the slow one
    m = bench.reduce_max(total_ms, world)
    q.put((rank, m, bench.whole_job_rate(2_000_000, 3, world, m)))
    dist.destroy_process_group()


def test_two_rank_reduction():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for rank, m, rate in out:
        assert m == 2000.0  # the slowest rank's time on every rank
        assert rate == pytest.approx(2 * 2_000_000 * 3 / 2.0)


def test_single_rank():
    import bench

    assert bench.reduce_max(5.0, 1) == 5.0
    assert bench.whole_job_rate(100, 2, 1, 1000.0) == 200.0
