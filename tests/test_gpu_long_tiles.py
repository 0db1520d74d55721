"""Matrices made of long dirty tiles, through the C ABI.

About 1,100 tiles that each span thousands of mostly empty rows, so that
kernel (c) re-arranges nearly all of them with whole blocks (several per
block), plus a run of 400,000 rows holding one tile's worth of entries: a tile
over more rows than the block's non-empty flag area holds, whose second pass
walks the row pointers again.  FP64 against the oracle's index artefacts and
y (both dirty-tile variants, two tile widths) and split into tile-range
shards; FP32 and a batch against the compensated bound of the
reduced-precision tests.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from test_gpu_batched import Batch, _C, _check_all  # noqa: E402
from test_gpu_parity import check_case  # noqa: E402
from test_gpu_reduced import _check, _run  # noqa: E402
from test_gpu_shards import _ntiles, _run_shards  # noqa: E402


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1504_06474_gb300 import _build
    _build.build()
    return torch.device("cuda:0")


def long_tile_matrix(seed: int = 21):
    """2,000 dense rows, 2.2 M rows with one non-empty row in twelve (1-4
    entries: tiles of 480 entries over ~2,400 rows), 400,000 rows holding 120
    rows of 4 entries, then 50,000 rows like the second part."""
    rng = np.random.Generator(np.random.PCG64(seed))
    head = rng.integers(20, 40, 2000)
    sparse = np.where(rng.random(2_200_000) < 1.0 / 12, rng.integers(1, 5, 2_200_000), 0)
    run = np.zeros(400_000, np.int64)
    run[rng.choice(400_000, 120, replace=False)] = 4
    tail = np.where(rng.random(50_000) < 1.0 / 12, rng.integers(1, 5, 50_000), 0)
    lens = np.concatenate([head, sparse, run, tail])
    A = synth.from_lengths(lens, 50_000, seed=seed)
    return A, synth.sym_vector(A.n, seed=seed)


def _spans(A, L):
    toff = oracle.tile_offsets(A.row_ptr, L)
    return np.diff(toff)


def test_the_matrix_has_what_the_tests_need():
    A, _ = long_tile_matrix()
    span = _spans(A, 480)
    assert (span > 1024).sum() > 900           # long tiles for whole blocks, several per block
    assert span.max() > 100_000                # past the flag area of FP64 and FP32 blocks


@pytest.mark.parametrize("W", [0, 31])
def test_long_tiles_f64(dev, W):
    A, x = long_tile_matrix()
    check_case(dev, A.row_ptr, A.col, A.val, x, A.n, W=W)


def test_long_tiles_f32(dev):
    A, x = long_tile_matrix()
    v32, x32 = A.val.astype(np.float32), x.astype(np.float32)
    y = _run(dev, A, torch.as_tensor(v32, device=dev), torch.as_tensor(x32, device=dev), "f32")
    _check(A, x, v32.astype(np.float64), x32.astype(np.float64), y, "long tiles f32")


def test_long_tiles_in_a_batch(dev):
    A, x = long_tile_matrix()
    small = [synth.batch_matrix(s) for s in synth.batch_specs(6, seed=22, m_lo=40, m_hi=20000)]
    b = Batch(small[:3] + [(A, x)] + small[3:], dev)
    C = _C()
    opts = C.make_opts()
    ws = b.run(opts)
    assert C.ssspmv_device_status(ws) == 0
    _check_all(b, opts)


def test_long_tiles_in_four_shards(dev):
    from paper_1504_06474_gb300 import api
    A, x = long_tile_matrix()
    y = _run_shards(dev, A, x, api.split_tiles(_ntiles(A), 4))
    yref, s = oracle.spmv_dot2(A.row_ptr, A.col, A.val, x)
    assert np.all(np.abs(y - yref) <= 1e-13 * s)
    assert np.all(y[s == 0] == 0.0)
