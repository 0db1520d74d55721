"""bench.py's host logic on CPU: the replica coordination (two ranks in a gloo
process group agree on the slowest rank's time, and the whole-job throughput
counts every replica's products: the N-GPU run is N independent replicas, no
collective on the data path), the byte counts behind the GB/s figures, and the
rule that an ncu traffic record only holds for the sources it came from."""
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


def test_byte_counts():
    import bench
    # stencil160: nnz (8 + 4) + (m + 1) 4 + m 8 + n 8 = 1,392,504,228 B (x once)
    m = n = 4_096_000
    nnz = 109_215_352
    assert bench.algorithmic_bytes(m, n, nnz) == 1_392_504_228
    # FP32 values and vectors; BF16 values with FP32 vectors
    assert bench.algorithmic_bytes(m, n, nnz, val_bytes=4, y_bytes=4, x_bytes=4) == (
        nnz * 8 + (m + 1) * 4 + m * 4 + n * 4)
    assert bench.algorithmic_bytes(m, n, nnz, val_bytes=2, y_bytes=4, x_bytes=4) == (
        nnz * 6 + (m + 1) * 4 + m * 4 + n * 4)
    # the paper's numerator counts x once per entry: (m+1+nnz) idx + (2 nnz + m) val
    assert bench.paper_bytes(m, nnz) == (m + 1 + nnz) * 4 + (2 * nnz + m) * 8


def test_traffic_record_follows_the_sources(tmp_path, monkeypatch):
    import json
    import bench
    rec = {"records": [{"kernel": "segsum_kernel", "workload": "w", "dram_bytes_per_launch": 7,
                        "source_digest": bench.source_digest()}]}
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # the digest is computed over the package sources, found from ROOT too
    monkeypatch.setattr(bench, "source_digest", lambda: rec["records"][0]["source_digest"])
    assert bench.ncu_traffic("segsum_kernel", "w") == 7
    assert bench.ncu_traffic("segsum_kernel", "other") is None
    monkeypatch.setattr(bench, "source_digest", lambda: "0" * 16)   # sources changed since
    assert bench.ncu_traffic("segsum_kernel", "w") is None

