"""y = alpha A x + beta y (ssspmv_csr_f64_axpby, ssspmv_plan_execute_axpby)
against the oracle: |y - (alpha yref + beta y_old)| <= |alpha| 1e-13 s +
2u (|alpha yref| + |beta y_old|) per row; y is not read when beta == 0."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-13
U = 2.0 ** -53


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1504_06474_gb300 import _build
    _build.build()
    return torch.device("cuda:0")


def _cases():
    yield synth.workload("uniform4096")
    lens = synth.random_lengths(15000, seed=41, mean=5.0, p_empty=0.4, p_long=0.001,
                                long_len=6000)
    A = synth.from_lengths(lens, 8000, seed=41)
    yield A, synth.sym_vector(A.n, seed=41)
    yield synth.rmat(14, 16, (0.57, 0.19, 0.19), seed=42, inject_len=3000), \
        synth.sym_vector(1 << 14, seed=42)


def _check(y, yref, s, y_old, alpha, beta):
    ref = alpha * yref + (beta * y_old if beta != 0 else 0.0)
    bound = abs(alpha) * TOL * s + 2 * U * (np.abs(alpha * yref) +
                                            (np.abs(beta * y_old) if beta != 0 else 0.0))
    assert np.all(np.isfinite(y))
    assert np.all(np.abs(y - ref) <= bound + 1e-300)


@pytest.mark.parametrize("alpha,beta", [(1.0, 0.0), (2.5, 0.0), (-0.5, 1.25), (0.0, 3.0)])
@pytest.mark.parametrize("variant,W", [(0, 0), (1, 27), (2, 15), (3, 0)])
def test_axpby(dev, alpha, beta, variant, W):
    from paper_1504_06474_gb300 import ssspmv as C
    rng = np.random.default_rng(3)
    for A, x in _cases():
        rp = torch.as_tensor(A.row_ptr, device=dev)
        col = torch.as_tensor(A.col, device=dev)
        val = torch.as_tensor(A.val, device=dev)
        xd = torch.as_tensor(x, device=dev)
        y_old = rng.uniform(-1, 1, A.m)
        y = torch.as_tensor(y_old if beta != 0 else np.full(A.m, np.nan), device=dev)
        opts = C.make_opts(W=W, variant=variant)
        ws = torch.empty(max(256, C.ssspmv_workspace_bytes(A.m, A.nnz, 8, opts)),
                         dtype=torch.uint8, device=dev)
        C.check(C.ssspmv_csr_f64_axpby(A.m, A.n, A.nnz, rp, col, val, xd, y, alpha, beta,
                                       opts=opts, workspace=ws), "axpby")
        assert C.ssspmv_device_status(ws) == 0
        yref, s = oracle.spmv_dot2(A.row_ptr, A.col, A.val, x)
        _check(y.cpu().numpy(), yref, s, y_old, alpha, beta)


def test_plan_axpby_iterations(dev):
    """A few steps of y <- 0.5 A x + 0.75 y through one plan."""
    from paper_1504_06474_gb300 import ssspmv as C
    A, x = next(iter(_cases()))
    rp = torch.as_tensor(A.row_ptr, device=dev)
    col = torch.as_tensor(A.col, device=dev)
    val = torch.as_tensor(A.val, device=dev)
    xd = torch.as_tensor(x, device=dev)
    y_h = np.zeros(A.m)
    y = torch.zeros(A.m, dtype=torch.float64, device=dev)
    plan = C.ssspmv_plan_create(A.m, A.n, A.nnz, rp, 8, None)
    try:
        yref, s = oracle.spmv_dot2(A.row_ptr, A.col, A.val, x)
        for _ in range(3):
            C.check(C.ssspmv_plan_execute_axpby(plan, col, val, xd, y, 0.5, 0.75), "execute")
            y_old = y_h
            y_h = y.cpu().numpy()
            _check(y_h, yref, s, y_old, 0.5, 0.75)
    finally:
        C.ssspmv_plan_destroy(plan)
