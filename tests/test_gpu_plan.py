"""Plans (kernel (a) once, kernels (b) and (c) per execution) and the
library-owned workspace, through the C ABI, against the CPU oracle and
against the single call bit for bit (same tile shape, same arithmetic)."""
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


def _C():
    from paper_1504_06474_gb300 import ssspmv
    return ssspmv


def _structure(seed):
    lens = synth.random_lengths(20000, seed=seed, mean=7.0, p_empty=0.25, p_long=0.0005,
                                long_len=4000)
    return synth.from_lengths(lens, 6000, seed=seed)


def _single_f64(C, A, col, val, x, opts):
    y = torch.empty(A.m, dtype=torch.float64, device=x.device)
    ws = torch.empty(C.ssspmv_workspace_bytes(A.m, A.nnz, 8, opts), dtype=torch.uint8,
                     device=x.device)
    C.check(C.ssspmv_csr_f64(A.m, A.n, A.nnz, A.rp_d, col, val, x, y, opts=opts, workspace=ws),
            "ssspmv_csr_f64")
    return y


@pytest.mark.parametrize("variant", [1, 2])
def test_plan_f64_many_executions(dev, variant):
    C = _C()
    A = _structure(21)
    A.rp_d = torch.as_tensor(A.row_ptr, device=dev)
    col = torch.as_tensor(A.col, device=dev)
    opts = C.make_opts(variant=variant)
    plan = C.ssspmv_plan_create(A.m, A.n, A.nnz, A.rp_d, 8, opts)
    try:
        rng = np.random.default_rng(5)
        for k in range(4):   # new values and x on the same pattern every time
            val_h = rng.uniform(-1, 1, A.nnz)
            x_h = rng.uniform(-1, 1, A.n)
            val = torch.as_tensor(val_h, device=dev)
            x = torch.as_tensor(x_h, device=dev)
            y = torch.full((A.m,), float("nan"), dtype=torch.float64, device=dev)
            C.check(C.ssspmv_plan_execute(plan, col, val, x, y), "ssspmv_plan_execute")
            yh = y.cpu().numpy()
            yref, s = oracle.spmv_dot2(A.row_ptr, A.col, val_h, x_h)
            assert np.all(np.abs(yh - yref) <= TOL * s)
            assert np.all(yh[s == 0] == 0.0)
            single = _single_f64(C, A, col, val, x, opts).cpu().numpy()
            assert np.array_equal(yh, single)
        ptr, nbytes = C.ssspmv_plan_workspace(plan)
        assert ptr and nbytes >= C.ssspmv_workspace_bytes(A.m, A.nnz, 8, opts)
        assert C.ssspmv_device_status(ptr, nbytes) == 0
    finally:
        C.ssspmv_plan_destroy(plan)


def test_plan_with_caller_workspace_and_f32(dev):
    C = _C()
    A = _structure(22)
    rp = torch.as_tensor(A.row_ptr, device=dev)
    col = torch.as_tensor(A.col, device=dev)
    val32 = torch.as_tensor(A.val.astype(np.float32), device=dev)
    x_h = synth.sym_vector(A.n, seed=22).astype(np.float32)
    x32 = torch.as_tensor(x_h, device=dev)
    ws = torch.empty(C.ssspmv_workspace_bytes(A.m, A.nnz, 4, None), dtype=torch.uint8,
                     device=dev)
    plan = C.ssspmv_plan_create(A.m, A.n, A.nnz, rp, 4, None, workspace=ws)
    try:
        y = torch.empty(A.m, dtype=torch.float32, device=dev)
        C.check(C.ssspmv_plan_execute(plan, col, val32, x32, y), "ssspmv_plan_execute")
        y2 = torch.empty(A.m, dtype=torch.float32, device=dev)
        ws2 = torch.empty_like(ws)
        C.check(C.ssspmv_csr_f32(A.m, A.n, A.nnz, rp, col, val32, x32, y2, workspace=ws2),
                "ssspmv_csr_f32")
        assert np.array_equal(y.cpu().numpy(), y2.cpu().numpy())
        ptr, _ = C.ssspmv_plan_workspace(plan)
        assert ptr == ws.data_ptr()
    finally:
        C.ssspmv_plan_destroy(plan)


def test_plan_timer_and_full_size_stencil(dev):
    C = _C()
    A, x_h = synth.workload("stencil100")
    rp = torch.as_tensor(A.row_ptr, device=dev)
    col = torch.as_tensor(A.col, device=dev)
    val = torch.as_tensor(A.val, device=dev)
    x = torch.as_tensor(x_h, device=dev)
    y = torch.empty(A.m, dtype=torch.float64, device=dev)
    plan = C.ssspmv_plan_create(A.m, A.n, A.nnz, rp, 8, None)
    timer = C.ssspmv_timer_create(3)
    try:
        for _ in range(3):
            C.check(C.ssspmv_plan_execute(plan, col, val, x, y, timer=timer), "execute")
        t = C.ssspmv_timer_read(timer, 3)
        assert len(t) == 3 and all(v[1] > 0 and v[3] >= v[1] for v in t)
        # rows sampled across the matrix against the oracle's row sums
        idx = np.linspace(0, A.m - 1, 4001).astype(np.int64)
        yref, s = oracle.spmv_dot2(A.row_ptr, A.col, A.val, x_h)
        yh = y.cpu().numpy()
        assert np.all(np.abs(yh[idx] - yref[idx]) <= TOL * s[idx])
        assert np.all(np.abs(yh - yref) <= TOL * s)
    finally:
        C.ssspmv_timer_destroy(timer)
        C.ssspmv_plan_destroy(plan)


def test_library_owned_workspace(dev):
    C = _C()
    A = _structure(23)
    rp = torch.as_tensor(A.row_ptr, device=dev)
    col = torch.as_tensor(A.col, device=dev)
    val = torch.as_tensor(A.val, device=dev)
    x_h = synth.sym_vector(A.n, seed=23)
    x = torch.as_tensor(x_h, device=dev)
    ref = _single_f64(C, type("A", (), dict(m=A.m, n=A.n, nnz=A.nnz, rp_d=rp)), col, val, x,
                      None).cpu().numpy()
    s1 = torch.cuda.Stream(dev)
    s2 = torch.cuda.Stream(dev)
    torch.cuda.synchronize()   # inputs were copied on the default stream
    ys = []
    for s in (s1, s2, s1):
        y = torch.empty(A.m, dtype=torch.float64, device=dev)
        with torch.cuda.stream(s):
            C.check(C.ssspmv_csr_f64(A.m, A.n, A.nnz, rp, col, val, x, y, workspace=None,
                                     stream=s), "ssspmv_csr_f64")
        ys.append((s, y))
    torch.cuda.synchronize()
    for _, y in ys:
        assert np.array_equal(y.cpu().numpy(), ref)
    p1, b1 = C.ssspmv_cached_workspace(s1)
    p2, b2 = C.ssspmv_cached_workspace(s2)
    assert p1 and p2 and p1 != p2 and p1 % 256 == 0
    assert b1 >= C.ssspmv_workspace_bytes(A.m, A.nnz, 8, None)
    assert C.ssspmv_device_status(p1, b1, stream=s1) == 0
    # a larger problem on the same stream grows the cached buffer
    big = synth.from_lengths(np.full(60000, 9), 6000, seed=3)
    rpb = torch.as_tensor(big.row_ptr, device=dev)
    colb = torch.as_tensor(big.col, device=dev)
    valb = torch.as_tensor(big.val, device=dev)
    xb_h = synth.sym_vector(big.n, seed=3)
    xb = torch.as_tensor(xb_h, device=dev)
    yb = torch.empty(big.m, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    with torch.cuda.stream(s1):
        C.check(C.ssspmv_csr_f64(big.m, big.n, big.nnz, rpb, colb, valb, xb, yb, workspace=None,
                                 stream=s1), "grow")
    torch.cuda.synchronize()
    yref, s = oracle.spmv_dot2(big.row_ptr, big.col, big.val, xb_h)
    assert np.all(np.abs(yb.cpu().numpy() - yref) <= TOL * s)
    _, b1b = C.ssspmv_cached_workspace(s1)
    assert b1b >= C.ssspmv_workspace_bytes(big.m, big.nnz, 8, None)
    C.ssspmv_release_workspaces()
    with pytest.raises(C.SsspmvError):
        C.ssspmv_cached_workspace(s1)


def test_spread_flag_across_calls_and_plans(dev):
    """Kernel (b)'s schedule flag lives in the workspace: kernel (a) sets it on
    a matrix with runs of empty rows (R-MAT scale 20, S = 1: shares of about
    ten bunches), kernel (c) clears it, and a plan keeps the one its creation
    set.  One workspace serves a flagged and an unflagged matrix in turn, and
    a plan executes several times; y is exact every time and the same bit for
    bit whatever the schedule."""
    C = _C()
    R, xr = synth.workload("rmat20")
    U, xu = synth.workload("uniform4096")
    opts = C.make_opts(S=1)
    nbytes = max(C.ssspmv_workspace_bytes(M.m, M.nnz, 8, opts) for M in (R, U))
    ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    dev_of = lambda M, x: [torch.as_tensor(a, device=dev) for a in (M.row_ptr, M.col, M.val, x)]
    Rd, Ud = dev_of(R, xr), dev_of(U, xu)
    refs = {id(R): oracle.spmv_dot2(R.row_ptr, R.col, R.val, xr),
            id(U): oracle.spmv_dot2(U.row_ptr, U.col, U.val, xu)}
    first = {}
    for M, (rp, col, val, x) in ((R, Rd), (U, Ud), (R, Rd), (R, Rd), (U, Ud)):
        y = torch.full((M.m,), float("nan"), dtype=torch.float64, device=dev)
        C.check(C.ssspmv_csr_f64(M.m, M.n, M.nnz, rp, col, val, x, y, opts=opts, workspace=ws),
                "ssspmv_csr_f64")
        assert C.ssspmv_device_status(ws) == 0
        yh = y.cpu().numpy()
        yref, s = refs[id(M)]
        assert np.all(np.abs(yh - yref) <= TOL * s)
        if id(M) in first:
            assert np.array_equal(yh, first[id(M)])
        first.setdefault(id(M), yh)
    # a plan on the flagged matrix, executed after calls on the other one
    rp, col, val, x = Rd
    plan = C.ssspmv_plan_create(R.m, R.n, R.nnz, rp, 8, opts)
    try:
        for k in range(3):
            yu = torch.empty(U.m, dtype=torch.float64, device=dev)
            C.check(C.ssspmv_csr_f64(U.m, U.n, U.nnz, *Ud[:3], Ud[3], yu, opts=opts,
                                     workspace=ws), "ssspmv_csr_f64")
            y = torch.full((R.m,), float("nan"), dtype=torch.float64, device=dev)
            C.check(C.ssspmv_plan_execute(plan, col, val, x, y), "ssspmv_plan_execute")
            assert np.array_equal(y.cpu().numpy(), first[id(R)])
        ptr, nb = C.ssspmv_plan_workspace(plan)
        assert C.ssspmv_device_status(ptr, nb) == 0
    finally:
        C.ssspmv_plan_destroy(plan)
