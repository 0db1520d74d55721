"""bench.py's replica coordination on CPU: two ranks in a gloo process group
agree on the slowest rank's time, and the whole-job throughput counts every
replica's products (the N-GPU run is N independent replicas, no collective on
the data path)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(0.25 + 0.5 * rank)  # rank 1 is the slow one
        dist.barrier()
        out[rank] = t
    finally:
        dist.destroy_process_group()


def test_two_ranks_agree_on_the_slowest_time():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        assert dict(out) == {0: 0.75, 1: 0.75}


def test_single_process_and_throughput():
    import bench
    assert bench.max_over_ranks(1.5) == 1.5  # no process group: the value itself
    # 2 replicas x 10 steps x 1.3925 GB in the slowest rank's 5.6 ms
    v = bench.replica_throughput(1_392_504_228, 10, 2, 5.6e-3)
    assert v == pytest.approx(1_392_504_228 * 20 / 5.6e-3 / 1e9)
