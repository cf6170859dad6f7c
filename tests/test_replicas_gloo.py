"""The multi-GPU path is replicas only (the ePIE sweep does not shard): the
bench aggregates independent ranks as the units all ranks processed over the
slowest rank's time.  Checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rate, slowest = bench.replica_rate(units=1000 * (rank + 1), seconds=0.5 + rank)
        out.put((rank, rate, slowest))
    finally:
        dist.destroy_process_group()


def test_replica_rate_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # units 1000 + 2000 over the slowest rank's 1.5 s, the same on every rank
    for _, rate, slowest in res:
        assert slowest == 1.5 and abs(rate - 2000.0) < 1e-9


def test_replica_rate_without_process_group():
    import bench
    assert bench.replica_rate(300, 1.5) == (200.0, 1.5)
