"""Reduced-precision variants against the FP64 oracle.

ssspmv_csr_f32 (FP32 val, x, y) and ssspmv_csr_bf16f32 (BF16 val, FP32 x, y)
accumulate each segment as a compensated FP32 pair (TwoProduct + TwoSum).
Their error is checked against the FP64 oracle run on the rounded inputs,
which isolates accumulation error.  A compensated sum is as accurate as a
sum in twice the working precision rounded once (Ogita-Rump-Oishi 2005):
to first order its error is u |y| + n u^2 s, with n the row length and
s_i = sum_k |a_ik x_k|, and n u^2 <= u for every row here (n <= 2^24).  The
tests assert, on rows of every length,
    |y_i - yref_i| <= 2 u |yref_i| + 2 u s_i,   u = 2^-24,
which a plain FP32 running sum misses on long rows (its error grows like
sqrt(n) u s to n u s), and one row built so that only compensation gives
the exact sum: 1.0 followed by 2^20 entries of 2^-25, x = 1, whose sum
1 + 2^-5 is an FP32 number (each 2^-25 is below half an ulp of 1, so a
plain FP32 sum stays near 1).  The error against the oracle on the original
FP64 inputs (input rounding included) is printed.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def comp_bound(yref, s):
    """Error bound of the compensated FP32 products on rows of any length."""
    return 2 * U32 * np.abs(yref) + 2 * U32 * s


def absorbing_row(lead_pos: int = 0, m_extra: int = 2):
    """CSR with one row of 1.0 (at position lead_pos) and 2^20 entries of
    2^-25, all on column 0 (x = 1), plus m_extra short rows after it; the
    long row's exact sum is 1 + 2^-5."""
    n_small = 1 << 20
    vals = np.full(n_small + 1, 2.0 ** -25)
    vals[lead_pos] = 1.0
    extra = np.array([0.5, -0.25] * m_extra)[:m_extra]
    val = np.concatenate([vals, extra])
    rp = np.array([0, n_small + 1] + [n_small + 2 + i for i in range(m_extra)], np.int32)
    col = np.zeros(val.size, np.int32)
    return synth.CSR(len(rp) - 1, 1, rp, col, val), np.ones(1)


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1504_06474_gb300 import _build
    _build.build()
    return torch.device("cuda:0")


def _run(dev, A, val_dev, x_dev, kind, W=0, S=0):
    from paper_1504_06474_gb300 import ssspmv as C
    vb = {"f32": 4, "bf16": 2}[kind]
    opts = C.make_opts(W=W, S=S)
    rp = torch.as_tensor(A.row_ptr, device=dev)
    col = torch.as_tensor(A.col, device=dev)
    y = torch.full((A.m,), float("nan"), dtype=torch.float32, device=dev)
    ws = torch.empty(C.ssspmv_workspace_bytes(A.m, A.nnz, vb, opts), dtype=torch.uint8,
                     device=dev)
    fn = C.ssspmv_csr_f32 if kind == "f32" else C.ssspmv_csr_bf16f32
    C.check(fn(A.m, A.n, A.nnz, rp, col, val_dev, x_dev, y, opts=opts, workspace=ws),
            "ssspmv_csr_" + kind)
    assert C.ssspmv_device_status(ws) == 0
    return y.cpu().numpy().astype(np.float64)


def _check(A, x64, val_r, x_r, y, label):
    yref, s = oracle.spmv_dot2(A.row_ptr, A.col, val_r, x_r)
    bound = comp_bound(yref, s)
    err = np.abs(y - yref)
    bad = np.nonzero(~(err <= bound))[0]
    assert bad.size == 0, "%s rows %s err %s bound %s" % (label, bad[:5], err[bad[:5]], bound[bad[:5]])
    assert np.all(y[s == 0] == 0.0)
    y64, s64 = oracle.spmv_dot2(A.row_ptr, A.col, A.val, x64)
    nz = s64 > 0
    rel_acc = float(np.max(err[nz] / s[nz])) if nz.any() else 0.0
    rel_all = float(np.max(np.abs(y - y64)[nz] / s64[nz])) if nz.any() else 0.0
    print("%s: max |y-yref|/s on rounded inputs %.3e; vs FP64 inputs %.3e" % (label, rel_acc,
                                                                            rel_all))
    return rel_acc, rel_all


CASES = [
    ("uniform4096", None),
    ("random_empty", dict(m=20000, mean=8, p_empty=0.5)),
    ("long_rows", dict(m=3000, mean=30, p_empty=0.05, p_long=0.003, long_len=40000)),
]


def _matrix(name, spec):
    if spec is None:
        return synth.workload(name)
    lens = synth.random_lengths(spec["m"], seed=7, mean=spec["mean"], p_empty=spec["p_empty"],
                                p_long=spec.get("p_long", 0.0), long_len=spec.get("long_len", 0))
    A = synth.from_lengths(lens, 4000, seed=7)
    return A, synth.sym_vector(4000, seed=8)


@pytest.mark.parametrize("name,spec", CASES)
def test_f32_compensated(dev, name, spec):
    A, x = _matrix(name, spec)
    v32 = A.val.astype(np.float32)
    x32 = x.astype(np.float32)
    for W in (15, 27):
        for S in (0, 1):
            y = _run(dev, A, torch.as_tensor(v32, device=dev), torch.as_tensor(x32, device=dev),
                     "f32", W, S)
            _check(A, x, v32.astype(np.float64), x32.astype(np.float64), y,
                   "f32 %s W=%d S=%d" % (name, W, S))


@pytest.mark.parametrize("name,spec", CASES)
def test_bf16_values(dev, name, spec):
    A, x = _matrix(name, spec)
    vbf = torch.as_tensor(A.val).to(torch.bfloat16)
    x32 = x.astype(np.float32)
    v_r = vbf.to(torch.float64).numpy()
    for W in (0, 15, 27):  # 0: the default (27 for long_rows' 30 entries per row)
        y = _run(dev, A, vbf.to(dev).view(torch.int16), torch.as_tensor(x32, device=dev), "bf16",
                 W, 0)
        _check(A, x, v_r, x32.astype(np.float64), y, "bf16 %s W=%d" % (name, W))


def test_rmat22_all_precisions(dev):
    """The R-MAT workload with its 10^6-entry row in FP32 and BF16 storage."""
    A, x = synth.workload("rmat22")
    x32 = x.astype(np.float32)
    v32 = A.val.astype(np.float32)
    y = _run(dev, A, torch.as_tensor(v32, device=dev), torch.as_tensor(x32, device=dev), "f32")
    _check(A, x, v32.astype(np.float64), x32.astype(np.float64), y, "f32 rmat22")
    vbf = torch.as_tensor(A.val).to(torch.bfloat16)
    y = _run(dev, A, vbf.to(dev).view(torch.int16), torch.as_tensor(x32, device=dev), "bf16")
    _check(A, x, vbf.to(torch.float64).numpy(), x32.astype(np.float64), y, "bf16 rmat22")


EXACT_LONG_ROW = 1.0 + 2.0 ** -5


@pytest.mark.parametrize("lead_pos", [0, 7, 480 * 3 + 17])
def test_compensation_is_exact_on_an_absorbing_row(dev, lead_pos):
    """Only compensated accumulation returns 1 + 2^-5 for the row of 1.0 and
    2^20 entries of 2^-25 (within two FP32 ulps of 1; a plain FP32 sum loses
    hundreds of ulps), in FP32 and BF16-valued storage, for several tile
    shapes and bunch sizes."""
    A, x = absorbing_row(lead_pos)
    x32 = x.astype(np.float32)
    for kind in ("f32", "bf16"):
        if kind == "f32":
            vdev = torch.as_tensor(A.val.astype(np.float32), device=dev)
        else:
            vdev = torch.as_tensor(A.val).to(torch.bfloat16).to(dev).view(torch.int16)
        for W in (15, 27):
            for S in (0, 1, 3):
                y = _run(dev, A, vdev, torch.as_tensor(x32, device=dev), kind, W, S)
                assert abs(y[0] - EXACT_LONG_ROW) <= 2 * 2.0 ** -23, (kind, W, S, y[0])
                assert np.array_equal(y[1:], A.val[-2:])
