"""ssspmv_csr_f64_noalloc: the FP64 product for callers that cannot allocate
device memory (code handed only device pointers, with no allocator of its
own, or code that must not call cudaMalloc on its hot path).  Its workspace is
the library's fixed device array; the results must match the workspace entry
point ssspmv_csr_f64 within the parity tolerance, call after call (the array
keeps the previous call's contents).  This file is collected last so that a
failure here comes after every other test has run."""
import numpy as np
import pytest

import oracle
import synth
from paper_1504_06474_gb300 import _build
from paper_1504_06474_gb300 import ssspmv as C

TOL = 1e-13
FAKE = 0x7f0000000000  # never dereferenced


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return C._lib()


def test_rejects_problems_beyond_the_fixed_scratch(lib):
    # ~2^31 entries need far more than SSSPMV_NOALLOC_SCRATCH_BYTES of tiles:
    # rejected on the host before any device work
    big_m, big_nnz = 50_000_000, 2_000_000_000
    assert C.ssspmv_workspace_bytes(big_m, big_nnz, 8, None) > C.SSSPMV_NOALLOC_SCRATCH_BYTES
    rc = C.ssspmv_csr_f64_noalloc(big_m, big_m, big_nnz, FAKE, FAKE, FAKE, FAKE, FAKE)
    assert rc == C.SSSPMV_ETOOLARGE
    assert "scratch" in C.ssspmv_strerror(rc)
    assert C.ssspmv_csr_f64_noalloc(-1, 4, 0, FAKE, FAKE, FAKE, FAKE, FAKE) == C.SSSPMV_EINVAL


# the largest nnz whose workspace fits the fixed scratch with the default
# options (W = 15, 4 tiles per bunch): 12 bytes per tile (offset, info, dirty
# list entry) plus a 24-byte synchronizer record per bunch, each section
# 256-byte aligned
NOALLOC_MAX_NNZ = 223_671_840


def test_capacity_boundary(lib):
    cap = C.SSSPMV_NOALLOC_SCRATCH_BYTES
    assert C.ssspmv_workspace_bytes(4_000_000, NOALLOC_MAX_NNZ, 8, None) <= cap
    assert C.ssspmv_workspace_bytes(4_000_000, NOALLOC_MAX_NNZ + 1, 8, None) > cap
    # one entry more is rejected on the host, before any device work
    rc = C.ssspmv_csr_f64_noalloc(4_000_000, 4_000_000, NOALLOC_MAX_NNZ + 1, FAKE, FAKE, FAKE,
                                  FAKE, FAKE)
    assert rc == C.SSSPMV_ETOOLARGE


def test_same_option_verdicts_as_the_workspace_call(lib):
    # a tile shape that is not compiled in: EUNSUPPORTED, as ssspmv_csr_f64 says
    opts = C.make_opts(W=17)
    assert C.ssspmv_csr_f64_noalloc(100, 100, 1000, FAKE, FAKE, FAKE, FAKE, FAKE,
                                    opts=opts) == C.SSSPMV_EUNSUPPORTED
    assert C.ssspmv_csr_f64(100, 100, 1000, FAKE, FAKE, FAKE, FAKE, FAKE, opts=opts,
                            workspace=FAKE, ws_bytes=1 << 30) == C.SSSPMV_EUNSUPPORTED
    # a misaligned value array: EINVAL, nothing queued
    assert C.ssspmv_csr_f64_noalloc(100, 100, 1000, FAKE, FAKE, FAKE + 8, FAKE,
                                    FAKE) == C.SSSPMV_EINVAL


@pytest.mark.gpu
def test_matches_workspace_entry_point_on_consecutive_calls(lib):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1504_06474_gb300 import api
    dev = torch.device("cuda:0")
    A1, x1 = synth.workload("uniform4096")
    lens = synth.random_lengths(30000, seed=21, mean=10, p_empty=0.4, p_long=0.002,
                                long_len=20000)
    A2 = synth.from_lengths(lens, 6000, seed=21)
    x2 = synth.sym_vector(6000, seed=22)
    # two different problems back to back, then the first again: each call
    # finds the previous call's scratch contents
    for A, x in ((A1, x1), (A2, x2), (A1, x1)):
        Ad = api.to_device(A.row_ptr, A.col, A.val, A.n, dev)
        xd = torch.as_tensor(x, device=dev)
        y_ws = api.spmv_f64(Ad, xd)
        y_na = torch.full((A.m,), float("nan"), dtype=torch.float64, device=dev)
        rc = C.ssspmv_csr_f64_noalloc(A.m, A.n, A.nnz, Ad.row_ptr, Ad.col, Ad.val, xd, y_na)
        assert rc == C.SSSPMV_OK, C.ssspmv_strerror(rc)
        torch.cuda.synchronize()
        _, s = oracle.spmv_dot2(A.row_ptr, A.col, A.val, x)
        a, b = y_na.cpu().numpy(), y_ws.cpu().numpy()
        assert np.all(np.abs(a - b) <= TOL * s)
        assert np.all(a[s == 0] == 0.0)
