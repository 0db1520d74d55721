"""The seeded generators produce well-formed CSR with the stated shapes."""
import numpy as np

import synth


def _wellformed(A):
    rp = A.row_ptr
    assert rp[0] == 0 and np.all(np.diff(rp) >= 0) and rp[-1] == len(A.col) == len(A.val)
    assert A.col.min(initial=0) >= 0 and A.col.max(initial=0) < max(A.n, 1)
    d = np.diff(A.col.astype(np.int64))
    starts = np.zeros(len(A.col), dtype=bool)
    starts[rp[:-1][np.diff(rp) > 0]] = True
    # strictly increasing inside each row (sorted, no duplicates)
    assert np.all((d > 0) | starts[1:])


def test_uniform4096_shape():
    A = synth.uniform_rows(4096, 4096, 32, 0.05, seed=0)
    _wellformed(A)
    lens = np.diff(A.row_ptr)
    assert lens.max() <= 32
    assert np.count_nonzero(lens == 0) >= round(0.05 * 4096)
    assert 55_000 < A.nnz < 70_000
    B = synth.uniform_rows(4096, 4096, 32, 0.05, seed=0)
    assert np.array_equal(A.col, B.col) and np.array_equal(A.val, B.val)


def test_stencil_counts_and_values():
    A = synth.stencil27(7, 5, 4, seed=1)
    _wellformed(A)
    assert A.nnz == (3 * 7 - 2) * (3 * 5 - 2) * (3 * 4 - 2)
    rows = np.repeat(np.arange(A.m), np.diff(A.row_ptr))
    diag = A.col == rows
    assert np.all(A.val[diag] == 26.0)
    off = A.val[~diag]
    assert np.all(np.abs(off + 1.0) <= 0.01)
    assert np.count_nonzero(diag) == A.m


def test_rmat_small():
    A = synth.rmat(10, 8, seed=3, inject_len=500)
    _wellformed(A)
    assert A.m == 1024
    assert int(np.diff(A.row_ptr).max()) == 500
    assert np.all(np.abs(A.val) <= 1.0)


def test_vectors_deterministic():
    a = synth.sym_vector(1000, seed=4)
    b = synth.sym_vector(1000, seed=4)
    c = synth.sym_vector(1000, seed=5)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert a.min() >= -1.0 and a.max() < 1.0


def test_banded_exact_columns():
    A = synth.banded(50, 7, seed=4)
    for r in range(50):
        cols = A.col[A.row_ptr[r]:A.row_ptr[r + 1]]
        assert list(cols) == list(range(max(0, r - 7), min(49, r + 7) + 1))
    assert A.nnz == sum(min(49, r + 7) - max(0, r - 7) + 1 for r in range(50))


def test_range_rows_and_clipped_rmat():
    B = synth.range_rows(3000, 4, 40, seed=5)
    L = np.diff(B.row_ptr)
    assert L.min() >= 4 and L.max() <= 40
    for r in (0, 1234, 2999):
        c = B.col[B.row_ptr[r]:B.row_ptr[r + 1]]
        assert np.all(np.diff(c) > 0) and c.max() < 3000
    C = synth.rmat_clipped(1500, 8, seed=6)
    assert C.m == C.n == 1500 and C.col.max() < 1500 and np.all(np.diff(C.row_ptr) >= 0)
    C2 = synth.rmat_clipped(1500, 8, seed=6)
    assert np.array_equal(C.col, C2.col) and np.array_equal(C.val, C2.val)


def test_batch_recipe():
    sp = synth.batch_specs(512, seed=3)
    assert sp == synth.batch_specs(512, seed=3)
    ms = np.array([s[1] for s in sp])
    assert ms.min() >= 1000 and ms.max() <= 200000
    assert {s[0] for s in sp} == set(synth.BATCH_FAMILIES)
    assert all(8 <= s[2] <= 64 for s in sp if s[0] == "banded")
