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
