"""Seeded synthetic CSR inputs shared by the oracle, the tests and the bench.

This package only manufactures inputs.  It holds none of the SpMV arithmetic;
the CPU oracle (``oracle/``) and the CUDA path (``paper_1504_06474_gb300``)
both consume its arrays and share no other code.  The heavy generators are in
``synth.c`` (counter-based SplitMix64 randomness, so outputs are identical on
x86 and Arm and for any thread count); small test patterns are drawn with
numpy's PCG64 here.

Named workloads (the shapes of the paper's benchmark suite, Table 5, stood in
by synthetic matrices because the real collection is not available):

* ``uniform4096``  m = n = 4096, row length ~ U{0..32}, 5% of rows forced
  empty, sorted distinct uniform columns, val and x ~ U[-1, 1), seed 0.
* ``stencil160``   27-point stencil on a 160^3 grid (4,096,000 rows,
  109,215,352 nnz), diagonal 26.0, off-diagonals -1.0 + U[-0.01, 0.01),
  x ~ U[-1, 1), seed 1.
* ``stencil<k>``   the same stencil on a k^3 grid (smaller cases for profiling).
* ``rmat<k>``      the R-MAT recipe below at scale k, injected row 10^6 * 2^(k-22).
* ``rmat22``       R-MAT scale 22, edge factor 16, (0.57, 0.19, 0.19, 0.05),
  duplicates merged, self loops kept, one seeded row replaced by 1,000,000
  distinct uniform sorted columns, val and x ~ U[-1, 1), seed 2.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``libsynth.so`` in place (gcc, OpenMP).  Returns its path."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=gnu11",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i32, i64, u64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        lib.synth_u64.restype = u64
        lib.synth_u64.argtypes = [u64, u64, u64]
        lib.synth_unit.restype = f64
        lib.synth_unit.argtypes = [u64, u64, u64]
        lib.synth_sym_vector.restype = None
        lib.synth_sym_vector.argtypes = [i64, u64, u64, P]
        lib.synth_uniform_rows_ptr.restype = i64
        lib.synth_uniform_rows_ptr.argtypes = [i32, i32, f64, u64, P]
        lib.synth_fill_uniform.restype = None
        lib.synth_fill_uniform.argtypes = [i32, i32, P, u64, P, P]
        lib.synth_stencil27.restype = i64
        lib.synth_stencil27.argtypes = [i32, i32, i32, u64, P, P, P]
        lib.synth_rmat.restype = i64
        lib.synth_rmat.argtypes = [i32, i64, f64, f64, f64, u64, i64, P, P, P, i64, P]
        lib.synth_banded.restype = i64
        lib.synth_banded.argtypes = [i32, i32, u64, P, P, P]
        lib.synth_range_rows_ptr.restype = i64
        lib.synth_range_rows_ptr.argtypes = [i32, i32, i32, u64, P]
        lib.synth_blockdiag.restype = i64
        lib.synth_blockdiag.argtypes = [i32, i32, i32, u64, P, P, P]
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


@dataclass
class CSR:
    """A CSR matrix in host memory: int32 row_ptr[m+1], int32 col[nnz], f64 val[nnz]."""
    m: int
    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    name: str = ""
    note: str = ""

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1]) if self.m > 0 else 0


def sym_vector(n: int, seed: int, stream: int = 0) -> np.ndarray:
    """Dense f64 vector with entries uniform in [-1, 1)."""
    out = np.empty(max(n, 0), dtype=np.float64)
    if n > 0:
        _load().synth_sym_vector(n, seed, stream, _p(out))
    return out


def uniform_rows(m: int, n: int, maxlen: int = 32, empty_frac: float = 0.05,
                 seed: int = 0) -> CSR:
    lib = _load()
    row_ptr = np.empty(m + 1, dtype=np.int32)
    nnz = lib.synth_uniform_rows_ptr(m, maxlen, empty_frac, seed, _p(row_ptr))
    if nnz < 0:
        raise MemoryError("synth_uniform_rows_ptr failed")
    col = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float64)
    lib.synth_fill_uniform(m, n, _p(row_ptr), seed, _p(col), _p(val))
    return CSR(m, n, row_ptr, col, val, name="uniform%d" % m)


def stencil27(nx: int, ny: int, nz: int, seed: int = 1) -> CSR:
    lib = _load()
    m = nx * ny * nz
    row_ptr = np.empty(m + 1, dtype=np.int32)
    nnz = lib.synth_stencil27(nx, ny, nz, seed, _p(row_ptr), None, None)
    col = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float64)
    lib.synth_stencil27(nx, ny, nz, seed, _p(row_ptr), _p(col), _p(val))
    return CSR(m, m, row_ptr, col, val, name="stencil%dx%dx%d" % (nx, ny, nz))


def rmat(scale: int, edge_factor: int = 16, abc=(0.57, 0.19, 0.19), seed: int = 2,
         inject_len: int = 0) -> CSR:
    lib = _load()
    m = 1 << scale
    nedges = edge_factor * m
    cap = nedges + max(inject_len, 0)
    row_ptr = np.empty(m + 1, dtype=np.int32)
    col = np.empty(cap, dtype=np.int32)
    val = np.empty(cap, dtype=np.float64)
    inj = ctypes.c_int32(-1)
    nnz = lib.synth_rmat(scale, nedges, abc[0], abc[1], abc[2], seed, inject_len,
                         _p(row_ptr), _p(col), _p(val), cap, ctypes.byref(inj))
    if nnz < 0:
        raise MemoryError("synth_rmat failed")
    empty = int(np.count_nonzero(np.diff(row_ptr) == 0))
    note = "injected row %d; %d of %d rows empty (%.1f%%)" % (inj.value, empty, m, 100.0 * empty / m)
    return CSR(m, m, row_ptr, col[:nnz], val[:nnz], name="rmat%d" % scale, note=note)


def banded(m: int, k: int, seed: int) -> CSR:
    """Half-bandwidth k: row r holds columns max(0, r-k) .. min(m-1, r+k)."""
    lib = _load()
    row_ptr = np.empty(m + 1, dtype=np.int32)
    nnz = lib.synth_banded(m, k, seed, _p(row_ptr), None, None)
    if nnz < 0:
        raise MemoryError("synth_banded: nnz past int32")
    col = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float64)
    lib.synth_banded(m, k, seed, _p(row_ptr), _p(col), _p(val))
    return CSR(m, m, row_ptr, col, val, name="banded%d_k%d" % (m, k))


def range_rows(m: int, lo: int, hi: int, seed: int) -> CSR:
    """Row lengths uniform in {lo..hi}, sorted distinct uniform columns in [0, m)."""
    lib = _load()
    row_ptr = np.empty(m + 1, dtype=np.int32)
    nnz = lib.synth_range_rows_ptr(m, lo, hi, seed, _p(row_ptr))
    if nnz < 0:
        raise MemoryError("synth_range_rows_ptr: nnz past int32")
    col = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float64)
    lib.synth_fill_uniform(m, m, _p(row_ptr), seed, _p(col), _p(val))
    return CSR(m, m, row_ptr, col, val, name="uniform%d_%d_%d" % (m, lo, hi))


def rmat_clipped(m: int, edge_factor: int, seed: int) -> CSR:
    """R-MAT (0.57, 0.19, 0.19, 0.05) at scale ceil(log2 m), edge factor
    `edge_factor`, restricted to its leading m rows and columns."""
    scale = max(1, int(np.ceil(np.log2(max(m, 2)))))
    A = rmat(scale, edge_factor, (0.57, 0.19, 0.19), seed=seed)
    rp = A.row_ptr[: m + 1].astype(np.int64)
    col = A.col[: rp[-1]]
    val = A.val[: rp[-1]]
    keep = col < m
    kept = np.concatenate([[0], np.cumsum(keep, dtype=np.int64)])
    new_rp = kept[rp].astype(np.int32)
    return CSR(m, m, new_rp, col[keep].copy(), val[keep].copy(), name="rmat%d_ef%d" % (m, edge_factor))


def blockdiag(m: int, bmin: int, bmax: int, seed: int) -> CSR:
    """Dense diagonal blocks of sizes U{bmin..bmax}."""
    lib = _load()
    row_ptr = np.empty(m + 1, dtype=np.int32)
    nnz = lib.synth_blockdiag(m, bmin, bmax, seed, _p(row_ptr), None, None)
    if nnz < 0:
        raise MemoryError("synth_blockdiag: nnz past int32")
    col = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float64)
    lib.synth_blockdiag(m, bmin, bmax, seed, _p(row_ptr), _p(col), _p(val))
    return CSR(m, m, row_ptr, col, val, name="blockdiag%d" % m)


def long_rows(m: int, nlong: int, long_len: int, seed: int) -> CSR:
    """Short rows (lengths U{1..8}) with `nlong` seeded rows of `long_len`
    entries; sorted distinct uniform columns in [0, m)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lens = rng.integers(1, 9, size=m).astype(np.int64)
    lens[rng.choice(m, size=min(nlong, m), replace=False)] = min(long_len, m)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(lens, out=row_ptr[1:])
    if row_ptr[-1] > 0x7fffffff:
        raise MemoryError("long_rows: nnz past int32")
    row_ptr = row_ptr.astype(np.int32)
    nnz = int(row_ptr[-1])
    col = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float64)
    _load().synth_fill_uniform(m, m, _p(row_ptr), seed, _p(col), _p(val))
    return CSR(m, m, row_ptr, col, val, name="longrows%d" % m)


BATCH_FAMILIES = ("banded", "uniform", "rmat")


def batch_specs(count: int = 512, seed: int = 3, m_lo: int = 1000, m_hi: int = 200000):
    """The seeded recipe of a mixed batch: per matrix (family, m, parameter,
    seed) with m log-uniform in [m_lo, m_hi], the family drawn uniformly from
    banded (half-bandwidth k ~ U{8..64}), uniform random (row lengths
    U{4..40}) and R-MAT (edge factor 8, clipped to m)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    specs = []
    for i in range(count):
        fam = BATCH_FAMILIES[int(rng.integers(0, 3))]
        m = int(round(float(np.exp(rng.uniform(np.log(m_lo), np.log(m_hi))))))
        par = int(rng.integers(8, 65)) if fam == "banded" else (8 if fam == "rmat" else 0)
        specs.append((fam, m, par, int(seed) * 100003 + i))
    return specs


def batch_matrix(spec) -> tuple[CSR, np.ndarray]:
    """One matrix of a batch recipe with its x (U[-1, 1)), both FP64."""
    fam, m, par, s = spec
    if fam == "banded":
        A = banded(m, par, s)
    elif fam == "uniform":
        A = range_rows(m, 4, 40, s)
    else:
        A = rmat_clipped(m, par, s)
    return A, sym_vector(A.n, seed=s)


def workload(name: str) -> tuple[CSR, np.ndarray]:
    """The named workloads with their x vectors (see module docstring)."""
    if name == "uniform4096":
        A = uniform_rows(4096, 4096, 32, 0.05, seed=0)
        return A, sym_vector(A.n, seed=0)
    if name == "stencil160":
        A = stencil27(160, 160, 160, seed=1)
        A.name = "stencil160"
        return A, sym_vector(A.n, seed=1)
    if name.startswith("stencil") and name[7:].isdigit():
        k = int(name[7:])          # 27-point stencil on k^3 (profiling sizes)
        A = stencil27(k, k, k, seed=1)
        A.name = name
        return A, sym_vector(A.n, seed=1)
    if name == "rmat22":
        A = rmat(22, 16, (0.57, 0.19, 0.19), seed=2, inject_len=1_000_000)
        A.name = "rmat22"
        return A, sym_vector(A.n, seed=2)
    if name.startswith("rmat") and name[4:].isdigit():
        k = int(name[4:])          # the same recipe at scale k (the injected row scaled with m)
        A = rmat(k, 16, (0.57, 0.19, 0.19), seed=2, inject_len=(1_000_000 << k) >> 22)
        A.name = name
        return A, sym_vector(A.n, seed=2)
    raise KeyError(name)


# ---------------------------------------------------------------------------
# small structured patterns for tests (numpy PCG64, seeded)

def from_lengths(lengths, n: int, seed: int) -> CSR:
    """CSR with the given row lengths, sorted distinct uniform columns per row
    (columns with replacement when a row is longer than n), val ~ U[-1, 1)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lengths = np.asarray(lengths, dtype=np.int64)
    m = len(lengths)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(lengths, out=row_ptr[1:])
    nnz = int(row_ptr[-1])
    col = np.empty(nnz, dtype=np.int32)
    for r in range(m):
        k = int(lengths[r])
        if k == 0:
            continue
        if k <= n:
            c = np.sort(rng.choice(n, size=k, replace=False))
        else:
            c = np.sort(rng.integers(0, n, size=k))
        col[row_ptr[r]:row_ptr[r + 1]] = c
    val = rng.uniform(-1.0, 1.0, size=nnz)
    return CSR(m, n, row_ptr.astype(np.int32), col, val)


def random_lengths(m: int, seed: int, mean: float = 8.0, p_empty: float = 0.0,
                   p_long: float = 0.0, long_len: int = 2000) -> np.ndarray:
    """Row lengths: geometric-ish around `mean`, a fraction `p_empty` forced
    empty and a fraction `p_long` of rows made `long_len` long."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lens = rng.poisson(mean, size=m).astype(np.int64)
    if p_empty > 0:
        lens[rng.random(m) < p_empty] = 0
    if p_long > 0:
        lens[rng.random(m) < p_long] = long_len
    return lens
