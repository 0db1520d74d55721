"""One product split by tile ranges over two ranks, on the CPU: each gloo
rank computes its shard with the oracle's range-restricted row loop, the
ranks exchange their seam records (the partial sums of the rows cut at the
shard ends), and the library's host merge (ssspmv_seam_merge) adds each cut
row's partials in shard order.  The assembled y must equal the row loop's y
exactly (small integers).  No GPU is involved: this checks the split, the
exchange and the merge, which the GPU path shares."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _matrix(seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    lens = rng.integers(0, 50, size=3000)
    lens[:7] = 0                                        # leading empty rows
    lens[-5:] = 0                                       # trailing empty rows
    lens[rng.integers(10, 2990, size=4)] = 2500         # rows over several tiles
    rp = np.zeros(3001, np.int32)
    np.cumsum(lens, out=rp[1:])
    nnz = int(rp[-1])
    col = rng.integers(0, 200, size=nnz).astype(np.int32)
    val = rng.integers(-7, 8, size=nnz).astype(float)
    x = rng.integers(-7, 8, size=200).astype(float)
    return rp, col, val, x


def _shard_host(rank, world, rp, col, val, x, L):
    """The shard's y rows and seam record, computed by the oracle."""
    import oracle
    from paper_1504_06474_gb300 import api
    nnz = int(rp[-1])
    m = len(rp) - 1
    ntiles = (nnz + L - 1) // L
    t0, t1 = api.split_tiles(ntiles, world)[rank]
    B, E = min(t0 * L, nnz), min(t1 * L, nnz)
    toff = oracle.tile_offsets(rp, L)
    r_first, r_last = int(toff[t0]), int(toff[t1])
    part = oracle.spmv_range(rp, col, val, x, B, E)
    y = np.full(m, np.nan)
    if t0 == 0:
        y[:r_first] = 0.0
    y[r_first + 1:r_last] = part[r_first + 1:r_last]
    r2 = r_last if (r_first < r_last < m) else -1
    seam = np.array([r_first if r_first < m else -1, r2, 0, 0,
                     part[r_first] if r_first < m else 0.0, part[r2] if r2 >= 0 else 0.0])
    return y, seam


def _worker(rank, world, port, seed, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1504_06474_gb300 import api
        rp, col, val, x = _matrix(seed)
        y, seam = _shard_host(rank, world, rp, col, val, x, 480)
        seams = [torch.zeros(6, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(seams, torch.as_tensor(seam))
        rows, vals = api.merge_seams([s.numpy() for s in seams])
        parts = [torch.zeros(len(y), dtype=torch.float64) for _ in range(world)]
        dist.all_gather(parts, torch.as_tensor(y))
        if rank == 0:
            full = np.full(len(y), np.nan)
            for p in parts:
                p = p.numpy()
                have = ~np.isnan(p)
                assert not np.any(have & ~np.isnan(full)), "two shards own one row"
                full[have] = p[have]
            full[rows] = vals
            np.save(out, full)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("seed", [0, 1])
def test_two_rank_split_and_seam_exchange(tmp_path, seed):
    import oracle
    import torch.multiprocessing as mp
    out = str(tmp_path / "y.npy")
    mp.spawn(_worker, args=(2, _free_port(), seed, out), nprocs=2, join=True)
    y = np.load(out)
    rp, col, val, x = _matrix(seed)
    assert np.array_equal(y, oracle.spmv(rp, col, val, x))


def test_merge_rules():
    """Partials of one row from consecutive shards are summed in shard order;
    records out of order or with a bad status are refused."""
    from paper_1504_06474_gb300 import api
    from paper_1504_06474_gb300 import ssspmv as C
    recs = [np.array([0, 5, 0, 0, 1.5, 2.0]), np.array([5, -1, 0, 0, 0.25, 0.0]),
            np.array([5, 9, 0, 0, 0.125, 3.0]), np.array([9, 12, 0, 0, 1.0, 4.0])]
    rows, vals = api.merge_seams(recs)
    assert rows == [0, 5, 9, 12] and vals == [1.5, 2.375, 4.0, 4.0]
    with pytest.raises(C.SsspmvError):
        api.merge_seams([recs[2], recs[0]])
    bad = recs[1].copy()
    bad[2] = C.SSSPMV_DEV_RANGE
    with pytest.raises(C.SsspmvError):
        api.merge_seams([recs[0], bad])
