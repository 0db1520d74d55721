"""Parity of the CUDA path with the CPU oracle, through the C ABI.

Floating point: every row satisfies |y_i - yref_i| <= 1e-13 * s_i with yref
the oracle's compensated (Dot2) row sum and s_i = sum_k |a_ik x_k|; rows with
s_i = 0 must be exactly 0.  Integer artefacts (tile offsets, raw segment
descriptors, dirty flags, segment counts, synchronizer rows) must match the
oracle's independent derivations bit for bit.
"""
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


def _api():
    from paper_1504_06474_gb300 import api, ssspmv
    return api, ssspmv


def check_case(dev, row_ptr, col, val, x, n, W=0, S=0, expect_exact=None, variant=None,
               block_warps=0):
    """Runs both dirty-tile variants (speculative + calibration, and exact
    stores in kernel (b)) unless one is given; returns the last result."""
    _, C = _api()
    variants = [C.VARIANT_SPECULATIVE, C.VARIANT_EXACT] if variant is None else [variant]
    out = None
    for v in variants:
        out = _check_one(dev, row_ptr, col, val, x, n, W, S, expect_exact, v, block_warps)
    return out


def _check_one(dev, row_ptr, col, val, x, n, W, S, expect_exact, variant, block_warps=0):
    api, C = _api()
    A = api.to_device(row_ptr, col, val, n, dev)
    xd = torch.as_tensor(x, dtype=torch.float64, device=dev)
    opts = C.make_opts(W=W, S=S, variant=variant, block_warps=block_warps)
    out = api.spmv_f64_debug(A, xd, opts)
    shape = out["shape"]
    L = shape["L"]
    yref, s = oracle.spmv_dot2(row_ptr, col, val, x)
    y = out["y"]
    bad = np.nonzero(~(np.abs(y - yref) <= TOL * s))[0]
    assert bad.size == 0, "rows %s: y=%s ref=%s s=%s (shape %s)" % (
        bad[:5], y[bad[:5]], yref[bad[:5]], s[bad[:5]], shape)
    assert np.all(y[s == 0] == 0.0)
    if expect_exact is not None:
        assert np.array_equal(y, expect_exact)
    # index artefacts, bit for bit
    toff = oracle.tile_offsets(row_ptr, L)
    assert np.array_equal(out["tile_offset"], toff)
    nt = shape["ntiles"]
    if nt:
        d = oracle.descriptors(row_ptr, L, toff)
        assert np.array_equal(out["desc"], d)
        dirty, nseg = oracle.tile_flags(row_ptr, L, toff)
        info = out["tile_info"]
        assert np.array_equal((info >> 31).astype(np.uint8), dirty)
        assert np.array_equal((info & 0x3FFFFFFF).astype(np.int32), nseg)
        resolved = ((info >> 30) & 1).astype(np.uint8)
        if variant == C.VARIANT_EXACT:
            assert np.array_equal(resolved, dirty)     # every dirty tile resolved in (b)
        else:
            assert not resolved.any()
        Sx = shape["S"]
        assert np.array_equal(out["sync_idx"], toff[np.arange(shape["nbunches"]) * Sx])
    return out


def test_paper_example_6x6(dev):
    rp = np.array([0, 3, 6, 8, 8, 9, 12], np.int32)
    col = np.array([0, 2, 5, 0, 1, 2, 2, 4, 4, 2, 3, 4], np.int32)
    val = np.arange(3.0, 15.0)
    x = np.arange(1.0, 7.0)
    want = oracle.spmv(rp, col, val, x)
    for W in _api()[1].ssspmv_supported_w():
        check_case(dev, rp, col, val, x, 6, W=W, expect_exact=want)


def test_uniform4096_all_shapes(dev):
    A, x = synth.workload("uniform4096")
    for W in _api()[1].ssspmv_supported_w():
        for S in (0, 1, 2, 7):
            check_case(dev, A.row_ptr, A.col, A.val, x, A.n, W=W, S=S)


@pytest.mark.parametrize("bw", [1, 3, 8, 17, 64])
def test_block_warps(dev, bw):
    """Kernel (b) launched with fewer warps per block than it was compiled
    for, and with an over-large request (lowered to the most that fit), gives
    the same rows and index artefacts."""
    lens = synth.random_lengths(30000, seed=11, mean=6.0, p_empty=0.3, p_long=0.001,
                                long_len=3000)
    A = synth.from_lengths(lens, 5000, seed=11)
    x = synth.sym_vector(A.n, seed=11)
    for W in (0, 27):
        check_case(dev, A.row_ptr, A.col, A.val, x, A.n, W=W, block_warps=bw)


def test_spread_schedule(dev):
    """R-MAT at scale 20 with one tile per bunch: kernel (a) sees runs of 32
    empty rows and kernel (b) keeps only a third of each static share, the
    rest going to the ticket pool.  Every tile must be processed exactly once
    (the descriptor export is summed, so a second visit would show) and y and
    the index artefacts must match."""
    A, x = synth.workload("rmat20")
    lens = np.diff(np.asarray(A.row_ptr, np.int64))
    # precondition: all-empty aligned 32-row chunks among the rows the
    # partition kernel samples (the first of its four row chunks per thread)
    first = (min(A.m, 262144) // 32) * 32
    assert (lens[:first].reshape(-1, 32).sum(1) == 0).any()
    for W in (15, 21):
        check_case(dev, A.row_ptr, A.col, A.val, x, A.n, W=W, S=1)


@pytest.mark.parametrize("seed,mean,p_empty,p_long,long_len", [
    (1, 8, 0.5, 0.0, 0),        # half the rows empty: nearly every tile dirty
    (2, 3, 0.2, 0.0, 0),        # short rows: many segments per lane
    (3, 30, 0.05, 0.003, 20000),  # rows spanning many tiles and bunches
    (4, 1, 0.0, 0.0, 0),        # mostly single-entry rows
    (5, 60, 0.0, 0.0, 0),       # rows longer than a lane's run
])
def test_random_structures(dev, seed, mean, p_empty, p_long, long_len):
    lens = synth.random_lengths(20000, seed=seed, mean=mean, p_empty=p_empty, p_long=p_long,
                                long_len=long_len)
    A = synth.from_lengths(lens, 5000, seed=seed)
    x = synth.sym_vector(5000, seed=100 + seed)
    for W in (15, 27):
        for S in (0, 1, 3):
            check_case(dev, A.row_ptr, A.col, A.val, x, A.n, W=W, S=S)


@pytest.mark.parametrize("lens", [
    [0] * 1000 + [5] * 10 + [0] * 7,            # leading and trailing empty rows
    [100_000],                                  # one long row, many tiles
    [0, 0, 0],                                  # nnz = 0: y must be zeroed
    [1, 0, 2],                                  # fewer than 4 entries
    [3] * 7,                                    # 21 entries: ragged single tile
    [1] * 4000,                                 # a segment per entry
    [27] * 1000 + [0] + [27] * 1000,            # lanes aligned with rows, one empty
    [961, 0, 0, 961, 1],                        # rows exactly one tile long (W=31)
    [0] * 5 + [405] * 3 + [0] * 2 + [405],      # rows aligned with 15-wide tiles
    [3] * 100 + [0] * 5000 + [3] * 100,          # a dirty tile over 5,000 rows (block repair)
    ([2] * 240 + [0] * 1500) * 6 + [7] * 50,     # consecutive such tiles (one per block)
    [3] + [0] * 500 + [4] + [0] * 100 + [2] * 3 + [0] * 70,   # tiles over hundreds of rows
    ([0] * 40 + [1]) * 60 + [0] * 3000,         # sparse rows, long empty tail
    [500] + [0] * 2000 + [1] * 40 + [0] * 90 + [700],       # long rows around empty runs
])
def test_edge_structures(dev, lens):
    A = synth.from_lengths(lens, 64, seed=len(lens))
    x = synth.sym_vector(64, seed=9)
    for W in _api()[1].ssspmv_supported_w():
        for S in (0, 1, 2):
            check_case(dev, A.row_ptr, A.col, A.val, x, A.n, W=W, S=S)


@pytest.mark.parametrize("scale,inject", [(12, 0), (14, 3000), (16, 50000)])
def test_small_rmat(dev, scale, inject):
    """R-MAT's sparse tail: tiles spanning thousands of mostly empty rows."""
    A = synth.rmat(scale, 16, seed=scale, inject_len=inject)
    x = synth.sym_vector(A.n, seed=scale + 1)
    for W in (15, 27):
        for S in (0, 1, 5):
            check_case(dev, A.row_ptr, A.col, A.val, x, A.n, W=W, S=S)


def test_sparse_random(dev):
    lens = synth.random_lengths(60000, seed=13, mean=30, p_empty=0.95)
    A = synth.from_lengths(lens, 8000, seed=13)
    x = synth.sym_vector(8000, seed=14)
    for W in (15, 21, 31):
        check_case(dev, A.row_ptr, A.col, A.val, x, A.n, W=W, S=0)
        check_case(dev, A.row_ptr, A.col, A.val, x, A.n, W=W, S=2)


def test_duplicates_and_unsorted_columns(dev):
    rng = np.random.Generator(np.random.PCG64(5))
    lens = rng.integers(0, 40, size=3000)
    rp = np.zeros(3001, np.int32)
    np.cumsum(lens, out=rp[1:])
    nnz = int(rp[-1])
    col = rng.integers(0, 50, size=nnz).astype(np.int32)    # unsorted, repeated
    val = rng.uniform(-1, 1, nnz)
    x = rng.uniform(-1, 1, 50)
    check_case(dev, rp, col, val, x, 50)


def test_small_integers_exact(dev):
    rng = np.random.Generator(np.random.PCG64(8))
    lens = rng.integers(0, 70, size=5000)
    rp = np.zeros(5001, np.int32)
    np.cumsum(lens, out=rp[1:])
    nnz = int(rp[-1])
    col = rng.integers(0, 300, size=nnz).astype(np.int32)
    val = rng.integers(-8, 9, size=nnz).astype(float)
    x = rng.integers(-8, 9, size=300).astype(float)
    want = oracle.spmv(rp, col, val, x)   # exact: every partial sum is an integer < 2^53
    for W in _api()[1].ssspmv_supported_w():
        check_case(dev, rp, col, val, x, 300, W=W, S=1, expect_exact=want)


def test_nan_propagates_to_exactly_the_rows_that_use_it(dev):
    A, x = synth.workload("uniform4096")
    x = x.copy()
    x[123] = np.nan
    api, C = _api()
    Ad = api.to_device(A.row_ptr, A.col, A.val, A.n, dev)
    y = api.spmv_f64(Ad, torch.as_tensor(x, device=dev)).cpu().numpy()
    uses = np.zeros(A.m, bool)
    rows = np.repeat(np.arange(A.m), np.diff(A.row_ptr))
    uses[rows[A.col == 123]] = True
    assert np.array_equal(np.isnan(y), uses)


def test_deterministic(dev):
    lens = synth.random_lengths(50000, seed=11, mean=12, p_empty=0.3, p_long=0.001,
                                long_len=30000)
    A = synth.from_lengths(lens, 20000, seed=11)
    x = synth.sym_vector(20000, seed=12)
    api, C = _api()
    Ad = api.to_device(A.row_ptr, A.col, A.val, A.n, dev)
    xd = torch.as_tensor(x, device=dev)
    y1 = api.spmv_f64(Ad, xd).cpu().numpy()
    y2 = api.spmv_f64(Ad, xd).cpu().numpy()
    assert np.array_equal(y1.view(np.int64), y2.view(np.int64))


def test_host_buffer_entry_point(dev):
    A, x = synth.workload("uniform4096")
    api, C = _api()
    y_host = np.full(A.m, np.nan)
    nbytes = C.ssspmv_host_buffer_bytes(A.m, A.n, A.nnz)
    buf = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    rc = C.ssspmv_csr_f64_host(A.m, A.n, A.nnz, A.row_ptr, A.col, A.val, x, y_host,
                               dev_buffer=buf)
    assert rc == 0
    Ad = api.to_device(A.row_ptr, A.col, A.val, A.n, dev)
    y_dev = api.spmv_f64(Ad, torch.as_tensor(x, device=dev)).cpu().numpy()
    assert np.array_equal(y_host, y_dev)


def test_validate_csr(dev):
    api, C = _api()
    scratch = torch.zeros(4, dtype=torch.int32, device=dev)
    rp = torch.tensor([0, 2, 2, 5], dtype=torch.int32, device=dev)
    col = torch.tensor([0, 3, 1, 1, 2], dtype=torch.int32, device=dev)
    assert C.ssspmv_validate_csr(3, 4, 5, rp, col, scratch) == 0
    assert C.ssspmv_validate_csr(3, 3, 5, rp, col, scratch) == C.SSSPMV_EINVAL   # col 3 >= n
    bad_rp = torch.tensor([0, 3, 2, 5], dtype=torch.int32, device=dev)
    assert C.ssspmv_validate_csr(3, 4, 5, bad_rp, col, scratch) == C.SSSPMV_EINVAL
    assert C.ssspmv_validate_csr(3, 4, 4, rp, col, scratch) == C.SSSPMV_EINVAL   # rp[m] != nnz


# ---------------------------------------------------------------------------
# full-size workloads in the launch configuration the bench times (auto W, S)

@pytest.mark.parametrize("name", ["stencil160", "rmat22"])
def test_full_size_workloads(dev, name):
    A, x = synth.workload(name)
    api, C = _api()
    Ad = api.to_device(A.row_ptr, A.col, A.val, A.n, dev)
    xd = torch.as_tensor(x, device=dev)
    out = api.spmv_f64_debug(Ad, xd)
    yref, s = oracle.spmv_dot2(A.row_ptr, A.col, A.val, x)
    y = out["y"]
    assert np.all(np.abs(y - yref) <= TOL * s)
    assert np.all(y[s == 0] == 0.0)
    L = out["shape"]["L"]
    toff = oracle.tile_offsets(A.row_ptr, L)
    assert np.array_equal(out["tile_offset"], toff)
    dirty, nseg = oracle.tile_flags(A.row_ptr, L, toff)
    assert np.array_equal((out["tile_info"] >> 31).astype(np.uint8), dirty)
    assert np.array_equal((out["tile_info"] & 0x3FFFFFFF).astype(np.int32), nseg)
    # the descriptor on a sample of tiles spread over the matrix
    idx = np.unique(np.linspace(0, out["shape"]["ntiles"] - 1, 4001).astype(np.int64))
    d = oracle.descriptors(A.row_ptr, L, toff)
    assert np.array_equal(out["desc"][idx], d[idx])
    # the timed entry point gives the same y as the debug one
    y2 = api.spmv_f64(Ad, xd).cpu().numpy()
    assert np.array_equal(y, y2)


def test_stage_timer(dev):
    A, x = synth.workload("uniform4096")
    api, C = _api()
    Ad = api.to_device(A.row_ptr, A.col, A.val, A.n, dev)
    xd = torch.as_tensor(x, device=dev)
    timer = C.ssspmv_timer_create(3)
    try:
        opts = C.make_opts(timer=timer)
        ws = api.workspace_for(Ad, opts, device=dev)
        for _ in range(4):          # the fourth call exceeds the capacity: untimed
            api.spmv_f64(Ad, xd, opts=opts, workspace=ws)
        times = C.ssspmv_timer_read(timer, 8)
        assert len(times) == 3
        for a, b, c, whole in times:
            assert min(a, b, c) >= 0 and whole > 0
            assert abs((a + b + c) - whole) <= 1e-3 + 1e-3 * whole
        C.ssspmv_timer_reset(timer)
        assert C.ssspmv_timer_read(timer, 8) == []
    finally:
        C.ssspmv_timer_destroy(timer)


# ---------------------------------------------------------------------------
# the speculative stage's own output, before calibration (Sec. 3.2, Alg. 1)

def expected_speculative_rows(row_ptr, col, val, x, L, W, S, info):
    """Rows kernel (b) stores before calibration and the value each must hold,
    from the oracle's simulation of the speculative stage (Algorithm 1).

    Kernel (b) stores segment s of tile t at y[tile_offset[t] + s] -- on a
    dirty tile that is the paper's speculative, misplaced slot -- except:
    the bunch's first segment goes to the synchronizer record, and a tile's
    last segment whose row continues into the next tile is carried (the
    transmitter) and stored by the tile that finishes it.  Tiles resolved in
    kernel (b) (info bit 30) store every row of (start, stop) at its true
    row instead.  The oracle follows Algorithm 1, which resets the
    transmitter after a dirty tile (its checking stage adds that partial back
    when it moves it); kernel (b) carries it on, so a segment finished after
    a dirty tile holds the oracle's value plus the dirty tile's last partial,
    which the oracle leaves in that tile's last speculative slot."""
    rp = np.asarray(row_ptr, np.int64)
    m = len(rp) - 1
    nnz = int(rp[-1])
    toff = oracle.tile_offsets(row_ptr, L)
    _, nseg = oracle.tile_flags(row_ptr, L, toff)
    dirty = oracle.tile_flags(row_ptr, L, toff)[0]
    st = oracle.speculative_stage(row_ptr, col, val, x, 32, W, S)
    ys = st["y"]
    yfin = oracle.spmv(row_ptr, col, val, x)
    nt = len(nseg)
    rows, vals = [], []
    for t0 in range(0, nt, S):
        t1 = min(t0 + S, nt)
        rF = int(toff[t0])
        pending = 0.0   # a dirty tile's carried partial the oracle dropped
        for t in range(t0, t1):
            start, stop = int(toff[t]), int(toff[t + 1])
            e = min((t + 1) * L, nnz)
            cont = stop < m and rp[stop] < e
            ns = int(nseg[t])
            resolved = (int(info[t]) >> 30) & 1
            carried_on = ns == 1 and cont      # the tile lies inside one row
            if start != rF and not carried_on:
                rows.append(start)
                vals.append(ys[start] + pending)
            if not carried_on:
                pending = 0.0
            if resolved:
                for r in range(start + 1, stop):
                    rows.append(r)
                    vals.append(yfin[r])
            else:
                last = ns - 1 if cont else ns
                for s in range(1, last):
                    rows.append(start + s)
                    vals.append(ys[start + s])
            if cont and dirty[t]:
                pending += ys[start + ns - 1]
    return np.asarray(rows, np.int64), np.asarray(vals)


def _small_int_case(lens, n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    rp = np.zeros(len(lens) + 1, np.int32)
    np.cumsum(lens, out=rp[1:])
    nnz = int(rp[-1])
    col = rng.integers(0, n, size=nnz).astype(np.int32)
    val = rng.integers(-8, 9, size=nnz).astype(float)
    x = rng.integers(-8, 9, size=n).astype(float)
    return rp, col, val, x


@pytest.mark.parametrize("lens", [
    list(np.random.default_rng(1).integers(0, 70, size=5000)),      # short rows, some empty
    [3] + [0] * 500 + [4] + [0] * 100 + [2] * 3 + [0] * 70,         # tiles over hundreds of rows
    ([2] * 240 + [0] * 1500) * 6 + [7] * 50,                         # long dirty tiles
    [0] * 40 + [900] + [1, 0, 2, 0, 0, 5] * 200 + [1500] + [0, 3] * 300,  # dirty, then a long row
    [27] * 1000 + [0] + [27] * 1000,                                 # one empty row
])
def test_speculative_placement_before_calibration(dev, lens):
    """y after kernel (b), before kernel (c), slot by slot against the oracle's
    simulated speculative stage, bit for bit (small integers: every sum is
    exact in any order): on clean tiles segment s sits in row start + s, on
    dirty tiles the partials of the next non-empty rows sit in slots
    start + 1, ... (the paper's misplaced entries of Sec. 3.2), and kernel
    (b) writes no other row."""
    rp, col, val, x = _small_int_case(lens, 300, seed=len(lens))
    api, C = _api()
    A = api.to_device(rp, col, val, 300, dev)
    xd = torch.as_tensor(x, dtype=torch.float64, device=dev)
    for W in (15, 27):
        for S in (1, 2, 4):
            for variant in (C.VARIANT_SPECULATIVE, C.VARIANT_EXACT):
                out = api.spmv_f64_debug(A, xd, C.make_opts(W=W, S=S, variant=variant))
                L = out["shape"]["L"]
                rows, want = expected_speculative_rows(rp, col, val, x, L, W, S,
                                                       out["tile_info"])
                ys = out["y_spec"]
                written = np.zeros(len(rp) - 1, bool)
                written[rows] = True
                if variant == C.VARIANT_SPECULATIVE:
                    # kernel (b) writes exactly these rows (y started as NaN)
                    assert np.array_equal(~np.isnan(ys), written), (W, S, variant)
                bad = np.nonzero(ys[rows] != want)[0]
                assert bad.size == 0, (W, S, variant, rows[bad[:5]], ys[rows[bad[:5]]],
                                       want[bad[:5]])
