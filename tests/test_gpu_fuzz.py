"""Seeded fuzz of the whole path over many small random CSR structures:
row-length mixtures with runs of empty rows, rows over many tiles, rows
aligned with tiles, ragged last tiles, every compiled tile width, several
bunch sizes and both dirty-tile variants.  Each case is checked against the
oracle -- y exactly (small integers), tile offsets, descriptors, dirty flags
and segment counts bit for bit, the speculative stage's placement slot by
slot -- and split into shards whose merged y must be the same.  A second
fuzz draws larger, sparser structures (up to 300,000 rows, one non-empty row
in 3 to 400, long empty runs), so that most cases hold tiles over more than
1,024 rows, which kernel (c) re-arranges with whole blocks."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1504_06474_gb300 import _build
    _build.build()
    return torch.device("cuda:0")


def _case(rng):
    m = int(rng.integers(1, 2500))
    kind = int(rng.integers(0, 5))
    if kind == 0:      # short rows, many empty
        lens = rng.integers(0, 6, size=m) * (rng.random(m) > 0.6)
    elif kind == 1:    # runs of empty rows between short ones
        lens = np.where(rng.random(m) < 0.05, rng.integers(1, 30, size=m), 0)
    elif kind == 2:    # a few rows over many tiles
        lens = rng.integers(0, 20, size=m)
        lens[rng.integers(0, m, size=int(rng.integers(1, 4)))] = int(rng.integers(500, 6000))
    elif kind == 3:    # rows whose lengths are multiples of lane and tile sizes
        unit = int(rng.choice([15, 21, 27, 31, 480, 672]))
        lens = unit * rng.integers(0, 3, size=m)
    else:              # uniform
        lens = rng.integers(0, 60, size=m)
    lens = lens.astype(np.int64)
    if rng.random() < 0.3:
        lens[: int(rng.integers(1, 50))] = 0            # leading empty rows
    if rng.random() < 0.3:
        lens[-int(rng.integers(1, 50)):] = 0            # trailing empty rows
    rp = np.zeros(m + 1, np.int64)
    np.cumsum(lens, out=rp[1:])
    nnz = int(rp[-1])
    n = int(rng.integers(1, 400))
    col = rng.integers(0, n, size=nnz).astype(np.int32)
    val = rng.integers(-6, 7, size=nnz).astype(float)
    x = rng.integers(-6, 7, size=n).astype(float)
    return rp.astype(np.int32), col, val, x, n


def test_fuzz_single_calls_and_shards(dev):
    from paper_1504_06474_gb300 import api
    from paper_1504_06474_gb300 import ssspmv as C
    from test_gpu_parity import expected_speculative_rows
    rng = np.random.default_rng(2024)
    widths = C.ssspmv_supported_w()
    for case in range(300):
        rp, col, val, x, n = _case(rng)
        W = int(rng.choice(widths))
        S = int(rng.integers(0, 6))
        variant = int(rng.choice([C.VARIANT_SPECULATIVE, C.VARIANT_EXACT]))
        opts = C.make_opts(W=W, S=S, variant=variant)
        A = api.to_device(rp, col, val, n, dev)
        xd = torch.as_tensor(x, dtype=torch.float64, device=dev)
        out = api.spmv_f64_debug(A, xd, opts)
        want = oracle.spmv(rp, col, val, x)
        tag = (case, len(rp) - 1, int(rp[-1]), W, S, variant)
        assert np.array_equal(out["y"], want), tag
        L = out["shape"]["L"]
        toff = oracle.tile_offsets(rp, L)
        assert np.array_equal(out["tile_offset"], toff), tag
        if out["shape"]["ntiles"]:
            assert np.array_equal(out["desc"], oracle.descriptors(rp, L, toff)), tag
            dirty, nseg = oracle.tile_flags(rp, L, toff)
            info = out["tile_info"]
            assert np.array_equal((info >> 31).astype(np.uint8), dirty), tag
            assert np.array_equal((info & 0x3FFFFFFF).astype(np.int32), nseg), tag
            rows, vals = expected_speculative_rows(rp, col, val, x, L, W, out["shape"]["S"], info)
            assert np.array_equal(out["y_spec"][rows], vals), tag
        # the same product split into shards
        nt = out["shape"]["ntiles"]
        shards = int(rng.integers(1, 5))
        y = torch.full((A.m,), float("nan"), dtype=torch.float64, device=dev)
        seams = [api.spmv_f64_shard(A, xd, y, t0, t1, opts)
                 for t0, t1 in api.split_tiles(nt, shards)]
        rws, vls = api.merge_seams(seams)
        yh = y.cpu().numpy()
        yh[rws] = vls
        assert np.array_equal(yh, want), tag + (shards,)


def _sparse_case(rng, seed):
    import synth
    m = int(np.exp(rng.uniform(np.log(1000), np.log(300000))))
    p = float(np.exp(rng.uniform(np.log(1 / 400), np.log(1 / 3))))
    lens = np.where(rng.random(m) < p, rng.integers(1, 9, m), 0).astype(np.int64)
    if rng.random() < 0.3:                                        # a few dense rows
        lens[rng.integers(0, m, int(rng.integers(1, 20)))] = rng.integers(100, 3000)
    if rng.random() < 0.3:                                        # a long empty run
        a = int(rng.integers(0, m))
        lens[a:a + int(rng.integers(1000, 50000))] = 0
    if rng.random() < 0.3:
        lens[: int(rng.integers(1, 3000))] = 0
    if rng.random() < 0.3:
        lens[-int(rng.integers(1, 3000)):] = 0
    n = int(rng.integers(1, 5000))
    return synth.from_lengths(lens, n, seed=seed), synth.sym_vector(n, seed=seed + 1)


def test_fuzz_long_dirty_tiles(dev):
    from paper_1504_06474_gb300 import api
    from paper_1504_06474_gb300 import ssspmv as C
    from test_gpu_parity import check_case
    from test_gpu_reduced import _check, _run
    nlong = 0
    for case in range(150):
        rng = np.random.default_rng(9000 + case)
        A, x = _sparse_case(rng, 9000 + case)
        if A.nnz == 0:
            continue
        W = int(rng.choice([0, 21, 27, 31]))
        S = int(rng.choice([0, 1, 2, 5]))
        nlong += int((np.diff(oracle.tile_offsets(A.row_ptr, 32 * (W or 15))) > 1024).sum())
        check_case(dev, A.row_ptr, A.col, A.val, x, A.n, W=W, S=S)   # both variants
        if case % 3 == 0:
            v32, x32 = A.val.astype(np.float32), x.astype(np.float32)
            y = _run(dev, A, torch.as_tensor(v32, device=dev), torch.as_tensor(x32, device=dev),
                     "f32", W=W, S=S)
            _check(A, x, v32.astype(np.float64), x32.astype(np.float64), y, "case %d" % case)
        if case % 3 == 1:
            opts = C.make_opts(W=W, S=S)
            Ad = api.to_device(A.row_ptr, A.col, A.val, A.n, dev)
            xd = torch.as_tensor(x, dtype=torch.float64, device=dev)
            y = torch.full((A.m,), float("nan"), dtype=torch.float64, device=dev)
            nt = C.ssspmv_plan_shape(A.m, A.nnz, 8, opts)["ntiles"]
            seams = [api.spmv_f64_shard(Ad, xd, y, t0, t1, opts)
                     for t0, t1 in api.split_tiles(nt, int(rng.integers(2, 6)))]
            rws, vls = api.merge_seams(seams)
            yh = y.cpu().numpy()
            yh[rws] = vls
            yref, s = oracle.spmv_dot2(A.row_ptr, A.col, A.val, x)
            assert np.all(np.abs(yh - yref) <= 1e-13 * s), case
    assert nlong > 500  # the cases did exercise the whole-block path
