"""One product split by tile ranges (ssspmv_csr_f64_range) on the GPU: every
shard's interior rows, the seam partials merged across shards
(ssspmv_seam_merge), and the assembled y against the oracle -- exactly on
small integers, within 1e-13 * sum|a x| per row otherwise.  Two processes on
one GPU exchange their seam records over gloo, as ranks on separate GPUs
would (their kernels never wait on one another)."""
import os
import socket

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-13


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1504_06474_gb300 import _build
    _build.build()
    return torch.device("cuda:0")


def _small_int(seed, m=4000, n=300):
    rng = np.random.Generator(np.random.PCG64(seed))
    lens = rng.integers(0, 60, size=m)
    lens[:5] = 0
    lens[-9:] = 0
    lens[rng.integers(10, m - 10, size=3)] = 4000
    rp = np.zeros(m + 1, np.int32)
    np.cumsum(lens, out=rp[1:])
    nnz = int(rp[-1])
    col = rng.integers(0, n, size=nnz).astype(np.int32)
    val = rng.integers(-8, 9, size=nnz).astype(float)
    x = rng.integers(-8, 9, size=n).astype(float)
    return synth.CSR(m, n, rp, col, val), x


def _run_shards(dev, A, x, splits, opts=None):
    from paper_1504_06474_gb300 import api
    Ad = api.to_device(A.row_ptr, A.col, A.val, A.n, dev)
    xd = torch.as_tensor(x, dtype=torch.float64, device=dev)
    y = torch.full((A.m,), float("nan"), dtype=torch.float64, device=dev)
    seams = [api.spmv_f64_shard(Ad, xd, y, t0, t1, opts) for t0, t1 in splits]
    rows, vals = api.merge_seams(seams)
    if rows:
        y[torch.as_tensor(rows, dtype=torch.int64, device=dev)] = torch.as_tensor(
            vals, dtype=torch.float64, device=dev)
    return y.cpu().numpy()


def _ntiles(A, opts=None):
    from paper_1504_06474_gb300 import ssspmv as C
    return C.ssspmv_plan_shape(A.m, A.nnz, 8, opts)["ntiles"]


@pytest.mark.parametrize("shards", [1, 2, 3, 7])
def test_shards_small_integers_exact(dev, shards):
    from paper_1504_06474_gb300 import api
    for seed in (1, 2):
        A, x = _small_int(seed)
        want = oracle.spmv(A.row_ptr, A.col, A.val, x)
        nt = _ntiles(A)
        y = _run_shards(dev, A, x, api.split_tiles(nt, shards))
        assert np.array_equal(y, want), (seed, shards)
        # uneven cuts, an empty shard, a cut inside a long row
        rng = np.random.default_rng(seed)
        cuts = sorted(set([0, nt] + rng.integers(0, nt + 1, size=shards).tolist()))
        cuts = cuts[:1] + cuts[:]                             # an empty leading shard
        y = _run_shards(dev, A, x, list(zip(cuts[:-1], cuts[1:])))
        assert np.array_equal(y, want), (seed, shards, cuts)


@pytest.mark.parametrize("W,S", [(15, 0), (27, 1), (21, 3)])
def test_shards_random_structures(dev, W, S):
    from paper_1504_06474_gb300 import api
    from paper_1504_06474_gb300 import ssspmv as C
    lens = synth.random_lengths(30000, seed=W, mean=9, p_empty=0.4, p_long=0.002, long_len=20000)
    A = synth.from_lengths(lens, 6000, seed=W)
    x = synth.sym_vector(6000, seed=W + 1)
    opts = C.make_opts(W=W, S=S)
    yref, s = oracle.spmv_dot2(A.row_ptr, A.col, A.val, x)
    for shards in (2, 5):
        y = _run_shards(dev, A, x, api.split_tiles(_ntiles(A, opts), shards), opts)
        assert np.all(np.abs(y - yref) <= TOL * s)
        assert np.all(y[s == 0] == 0.0)


def test_rmat22_in_three_shards(dev):
    """The power-law benchmark graph split in three, in the launch
    configuration of the single call (automatic W, S and block shape)."""
    from paper_1504_06474_gb300 import api
    A, x = synth.workload("rmat22")
    y = _run_shards(dev, A, x, api.split_tiles(_ntiles(A), 3))
    yref, s = oracle.spmv_dot2(A.row_ptr, A.col, A.val, x)
    assert np.all(np.abs(y - yref) <= TOL * s)
    assert np.all(y[s == 0] == 0.0)


def test_bounds_that_do_not_match_row_ptr_are_flagged(dev):
    from paper_1504_06474_gb300 import api
    from paper_1504_06474_gb300 import ssspmv as C
    A, x = _small_int(3)
    Ad = api.to_device(A.row_ptr, A.col, A.val, A.n, dev)
    xd = torch.as_tensor(x, device=dev)
    y = torch.zeros(A.m, dtype=torch.float64, device=dev)
    nt = _ntiles(A)
    t0, t1 = nt // 3, 2 * nt // 3
    r0, r1 = C.ssspmv_range_bounds(A.m, A.nnz, Ad.row_ptr, t0, t1)
    ws = torch.empty(C.ssspmv_range_workspace_bytes(A.m, A.nnz, t0, t1, r0 + 1, r1),
                     dtype=torch.uint8, device=dev)
    seam = torch.zeros(C.SEAM_BYTES, dtype=torch.uint8, device=dev)
    C.check(C.ssspmv_csr_f64_range(A.m, A.n, A.nnz, Ad.row_ptr, Ad.col, Ad.val, xd, y, t0, t1,
                                   r0 + 1, r1, seam, workspace=ws), "range")
    rec = C.seams_from_bytes(seam.cpu().numpy().tobytes())[0]
    assert rec.status == C.SSSPMV_DEV_RANGE
    with pytest.raises(C.SsspmvError):
        api.merge_seams([np.array([rec.row[0], rec.row[1], rec.status, 0, rec.val[0],
                                   rec.val[1]])])


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1504_06474_gb300 import api
        dev = torch.device("cuda:0")
        lens = synth.random_lengths(50000, seed=31, mean=12, p_empty=0.3, p_long=0.001,
                                    long_len=30000)
        A = synth.from_lengths(lens, 9000, seed=31)
        x = synth.sym_vector(9000, seed=32)
        Ad = api.to_device(A.row_ptr, A.col, A.val, A.n, dev)
        xd = torch.as_tensor(x, device=dev)
        y = torch.full((A.m,), float("nan"), dtype=torch.float64, device=dev)
        t0, t1 = api.split_tiles(_ntiles(A), world)[rank]
        seam = api.spmv_f64_shard(Ad, xd, y, t0, t1)
        seams = [torch.zeros(6, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(seams, torch.as_tensor(seam))
        rows, vals = api.merge_seams([s.numpy() for s in seams])
        mine = y.cpu()
        parts = [torch.zeros(A.m, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(parts, mine)
        if rank == 0:
            full = np.full(A.m, np.nan)
            for p in parts:
                p = p.numpy()
                own = ~np.isnan(p)
                full[own] = p[own]          # seam rows are replaced below
            full[rows] = vals
            np.save(out, full)
    finally:
        dist.destroy_process_group()


def test_two_processes_exchange_seams_over_gloo(dev, tmp_path):
    import torch.multiprocessing as mp
    out = str(tmp_path / "y.npy")
    mp.spawn(_rank, args=(2, _free_port(), out), nprocs=2, join=True)
    y = np.load(out)
    lens = synth.random_lengths(50000, seed=31, mean=12, p_empty=0.3, p_long=0.001,
                                long_len=30000)
    A = synth.from_lengths(lens, 9000, seed=31)
    x = synth.sym_vector(9000, seed=32)
    yref, s = oracle.spmv_dot2(A.row_ptr, A.col, A.val, x)
    assert np.all(np.abs(y - yref) <= TOL * s)
    assert np.all(y[s == 0] == 0.0)
