"""The multi-process replica path of bench.py (one process per GPU, no data-
path collective) on CPU with the gloo backend, world size 2: ranks agree on
the max of their times after the barriers, the whole-job throughput counts
every rank's units, and only rank 0 reports."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    import bench
    d = bench.Dist(world, backend="gloo")
    try:
        d.barrier()
        t_mine = 100.0 + 50.0 * rank            # rank 1 is the slow one
        t_max = d.max(t_mine)
        d.barrier()
        value = bench.replica_throughput(d.world, 1.0e9, 10, t_max)
        q.put((rank, d.world, t_max, value, d.rank == 0))
    finally:
        d.close()


def test_two_replicas_max_time_and_aggregate_throughput():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, w, t_max, value, reports in out:
        assert w == 2
        assert t_max == 150.0                   # the slowest rank's time
        # 2 ranks x 1e9 units x 10 steps / 0.150 s
        assert value == pytest.approx(2 * 1.0e9 * 10 / 0.150)
        assert reports == (rank == 0)


def test_single_process_needs_no_process_group():
    os.environ.pop("WORLD_SIZE", None)
    import bench
    d = bench.Dist(1, backend="gloo")
    assert d.world == 1 and d.pg is None
    assert d.max(3.5) == 3.5
    assert bench.replica_throughput(1, 2.0, 5, 1000.0) == pytest.approx(10.0)
