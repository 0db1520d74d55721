"""Batched FP32 products through the C ABI: every matrix of a mixed batch
against the single FP32 call (bit for bit) and against the FP64 oracle on the
rounded inputs (the compensated-FP32 bound of the reduced-precision tests);
invalid descriptors, capacity overflow, and replay of a captured CUDA graph."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


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


def _mixed_batch():
    mats = [synth.batch_matrix(s) for s in synth.batch_specs(36, seed=11, m_lo=40, m_hi=30000)]
    lens = synth.random_lengths(5000, seed=12, mean=5.0, p_empty=0.5)
    A = synth.from_lengths(lens, 3000, seed=12)
    mats.append((A, synth.sym_vector(A.n, seed=12)))                     # half the rows empty
    lens = synth.random_lengths(400, seed=13, mean=4.0, p_long=0.003, long_len=30000)
    A = synth.from_lengths(lens, 40000, seed=13)
    mats.append((A, synth.sym_vector(A.n, seed=13)))                     # rows over many tiles
    E = synth.CSR(100, 10, np.zeros(101, np.int32), np.zeros(0, np.int32), np.zeros(0))
    mats.append((E, synth.sym_vector(10, seed=14)))                      # no entries at all
    Z = synth.CSR(0, 0, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    mats.append((Z, np.zeros(0)))                                        # no rows
    mats.append(absorbing_row())                                         # 1 + 2^20 * 2^-25
    return mats


class Batch:
    def __init__(self, mats, dev):
        C = _C()
        self.mats = mats
        self.rp, self.col, self.val, self.x, self.y, self.v64, self.x64 = [], [], [], [], [], [], []
        descs = []
        for A, x in mats:
            v32 = A.val.astype(np.float32)
            x32 = x.astype(np.float32)
            rp = torch.as_tensor(A.row_ptr, device=dev)
            col = torch.as_tensor(A.col, device=dev)
            val = torch.as_tensor(v32, device=dev)
            xd = torch.as_tensor(x32, device=dev)
            y = torch.full((A.m,), float("nan"), dtype=torch.float32, device=dev)
            self.rp.append(rp); self.col.append(col); self.val.append(val)
            self.x.append(xd); self.y.append(y)
            self.v64.append(v32.astype(np.float64)); self.x64.append(x32.astype(np.float64))
            descs.append((A.m, A.n, A.nnz, rp, col, val, xd, y))
        raw = np.frombuffer(C.batch_descriptors(descs), dtype=np.uint8).copy()
        self.desc = torch.as_tensor(raw, device=dev)
        self.total_nnz = sum(A.nnz for A, _ in mats)

    def run(self, opts=None, total_nnz=None, stream=None):
        C = _C()
        tn = self.total_nnz if total_nnz is None else total_nnz
        ws = torch.empty(C.ssspmv_batched_workspace_bytes(len(self.mats), tn, 4, opts),
                         dtype=torch.uint8, device=self.desc.device)
        rc = C.ssspmv_csr_batched_f32(len(self.mats), self.desc, tn, opts=opts, workspace=ws,
                                      stream=stream)
        C.check(rc, "ssspmv_csr_batched_f32")
        return ws


def absorbing_row():
    """One row of 1.0 then 2^20 entries of 2^-25 on column 0 (x = 1): its
    exact sum 1 + 2^-5 is returned only by compensated accumulation."""
    n_small = 1 << 20
    val = np.full(n_small + 1, 2.0 ** -25)
    val[0] = 1.0
    rp = np.array([0, n_small + 1], np.int32)
    return synth.CSR(1, 1, rp, np.zeros(val.size, np.int32), val), np.ones(1)


def _single_f32(i, b, opts):
    C = _C()
    A, _ = b.mats[i]
    y = torch.empty(A.m, dtype=torch.float32, device=b.desc.device)
    ws = torch.empty(max(C.ssspmv_workspace_bytes(A.m, A.nnz, 4, opts), 256), dtype=torch.uint8,
                     device=b.desc.device)
    C.check(C.ssspmv_csr_f32(A.m, A.n, A.nnz, b.rp[i], b.col[i], b.val[i], b.x[i], y, opts=opts,
                             workspace=ws), "ssspmv_csr_f32")
    return y.cpu().numpy()


def _check_all(b, opts, skip=()):
    for i, (A, _) in enumerate(b.mats):
        if i in skip or A.m == 0:
            continue
        y = b.y[i].cpu().numpy()
        assert np.array_equal(y, _single_f32(i, b, opts)), "matrix %d differs from the single call" % i
        yref, s = oracle.spmv_dot2(A.row_ptr, A.col, b.v64[i], b.x64[i])
        # the compensated bound of the reduced-precision tests, rows of any length
        bound = 2 * U32 * np.abs(yref) + 2 * U32 * s
        y64 = y.astype(np.float64)
        assert np.all(np.abs(y64 - yref) <= bound), "matrix %d outside the bound" % i
        assert np.all(y64[s == 0] == 0.0)


@pytest.mark.parametrize("W,S,variant", [(0, 0, 0), (27, 1, 0), (15, 7, 2), (21, 0, 2)])
def test_batch_matches_single_calls(dev, W, S, variant):
    C = _C()
    b = Batch(_mixed_batch(), dev)
    opts = C.make_opts(W=W, S=S, variant=variant)
    ws = b.run(opts)
    assert C.ssspmv_device_status(ws) == 0
    _check_all(b, opts)
    # the absorbing row (last matrix) is summed exactly, as in the single call
    assert abs(float(b.y[-1].cpu()[0]) - (1.0 + 2.0 ** -5)) <= 2 * 2.0 ** -23


def test_invalid_descriptor_is_skipped(dev):
    C = _C()
    mats = _mixed_batch()[:6]
    b = Batch(mats, dev)
    raw = b.desc.cpu().numpy().copy()
    raw[2 * 56 + 12: 2 * 56 + 16] = np.frombuffer(np.int32(1).tobytes(), np.uint8)  # reserved != 0
    b.desc = torch.as_tensor(raw, device=dev)
    ws = b.run()
    assert C.ssspmv_device_status(ws) == C.SSSPMV_DEV_BATCH
    assert torch.isnan(b.y[2]).all()                     # untouched
    _check_all(b, None, skip=(2,))


def test_capacity_overflow_computes_nothing(dev):
    C = _C()
    b = Batch(_mixed_batch()[:6], dev)
    ws = b.run(total_nnz=b.total_nnz // 4)
    assert C.ssspmv_device_status(ws) & C.SSSPMV_DEV_BATCH
    for y in b.y:
        assert torch.isnan(y).all()


def test_batch_replays_in_a_cuda_graph(dev):
    C = _C()
    b = Batch(_mixed_batch(), dev)
    ws = torch.empty(C.ssspmv_batched_workspace_bytes(len(b.mats), b.total_nnz, 4, None),
                     dtype=torch.uint8, device=dev)
    s = torch.cuda.Stream(dev)
    torch.cuda.synchronize()
    with torch.cuda.stream(s):  # warm-up outside capture (kernel attributes, occupancy)
        C.check(C.ssspmv_csr_batched_f32(len(b.mats), b.desc, b.total_nnz, workspace=ws,
                                         stream=s), "warm-up")
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        C.check(C.ssspmv_csr_batched_f32(len(b.mats), b.desc, b.total_nnz, workspace=ws,
                                         stream=s), "capture")
    for rep in range(2):
        rng = np.random.default_rng(40 + rep)
        for i, (A, _) in enumerate(b.mats):
            x32 = rng.uniform(-1, 1, A.n).astype(np.float32)
            b.x[i].copy_(torch.as_tensor(x32, device=dev))
            b.x64[i] = x32.astype(np.float64)
            b.y[i].fill_(float("nan"))
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        _check_all(b, None)
    assert C.ssspmv_device_status(ws) == 0
