"""Row-parallel CSR kernels (SSSPMV_VARIANT_ROWS: G lanes per row) against
the oracle's compensated row sums, through the C ABI, for every group size
and the automatic one; every row is written, empty rows as exact zeros."""
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


def _cases():
    yield "uniform4096", synth.workload("uniform4096")
    lens = synth.random_lengths(20000, seed=31, mean=6.0, p_empty=0.4)
    A = synth.from_lengths(lens, 5000, seed=31)
    yield "empty-rows", (A, synth.sym_vector(A.n, seed=31))
    lens = synth.random_lengths(3000, seed=32, mean=20.0, p_long=0.002, long_len=50000)
    A = synth.from_lengths(lens, 60000, seed=32)
    yield "long-rows", (A, synth.sym_vector(A.n, seed=32))
    A, x = synth.workload("stencil40")
    yield "stencil40", (A, x)


@pytest.mark.parametrize("G", [0, 1, 2, 4, 8, 16, 32])
def test_rows_variant(dev, G):
    from paper_1504_06474_gb300 import ssspmv as C
    for name, (A, x) in _cases():
        rp = torch.as_tensor(A.row_ptr, device=dev)
        col = torch.as_tensor(A.col, device=dev)
        val = torch.as_tensor(A.val, device=dev)
        xd = torch.as_tensor(x, device=dev)
        opts = C.make_opts(W=G, variant=C.VARIANT_ROWS)
        ws = torch.empty(C.ssspmv_workspace_bytes(A.m, A.nnz, 8, opts), dtype=torch.uint8,
                         device=dev)
        outs = []
        for _ in range(2):
            y = torch.full((A.m,), float("nan"), dtype=torch.float64, device=dev)
            C.check(C.ssspmv_csr_f64(A.m, A.n, A.nnz, rp, col, val, xd, y, opts=opts,
                                     workspace=ws), "rows G=%d %s" % (G, name))
            outs.append(y.cpu().numpy())
        assert np.array_equal(outs[0], outs[1])            # deterministic
        yref, s = oracle.spmv_dot2(A.row_ptr, A.col, A.val, x)
        y = outs[0]
        assert np.all(np.abs(y - yref) <= TOL * s), name
        assert np.all(y[s == 0] == 0.0), name
