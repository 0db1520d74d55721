"""CPU oracle for CSR SpMV by speculative segmented sum -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its binding) never touches it, and the two share no code: the oracle is plain
FP64 C (``oracle.c``) written from the paper's definitions, reached here
through ctypes.

Functions (each cites the passage it follows in ``oracle.c``):

* ``spmv(A, x)``             plain row loop, y = A x (Sec. 2.1)
* ``spmv_omp(A, x)``         same, rows split over OpenMP threads (Sec. 4.3)
* ``spmv_range(A, x, B, E)`` the row loop over the nonzeros [B, E) only
                             (one shard of a product split by ranges)
* ``spmv_dot2(A, x)``        compensated reference and per-row scale
                             sum_k |a_k x_k| (Ogita-Rump-Oishi Dot2)
* ``tile_offsets``, ``descriptors``, ``tile_flags``  index artefacts (Sec. 3.2)
* ``speculative_stage``, ``checking_stage``          Algorithm 1 and the
                             checking-prediction stage, simulated
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` in place: gcc -O2, no FP contraction, OpenMP."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               "-shared", "-fopenmp", "-std=gnu11", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i32, i64 = ctypes.c_int32, ctypes.c_int64
        lib.oracle_spmv_rowloop.restype = None
        lib.oracle_spmv_rowloop.argtypes = [i32, P, P, P, P, P]
        lib.oracle_spmv_rowloop_omp.restype = ctypes.c_int
        lib.oracle_spmv_rowloop_omp.argtypes = [i32, P, P, P, P, P, ctypes.c_int]
        lib.oracle_spmv_range.restype = None
        lib.oracle_spmv_range.argtypes = [i32, P, P, P, P, i64, i64, P]
        lib.oracle_spmv_dot2.restype = None
        lib.oracle_spmv_dot2.argtypes = [i32, P, P, P, P, P, P]
        lib.oracle_num_tiles.restype = i64
        lib.oracle_num_tiles.argtypes = [i64, i64]
        lib.oracle_tile_offsets.restype = None
        lib.oracle_tile_offsets.argtypes = [i32, i32, P, i32, P]
        lib.oracle_descriptors.restype = None
        lib.oracle_descriptors.argtypes = [i32, i32, P, i32, P, P]
        lib.oracle_tile_flags.restype = None
        lib.oracle_tile_flags.argtypes = [i32, i32, P, i32, P, P, P]
        lib.oracle_speculative_stage.restype = i64
        lib.oracle_speculative_stage.argtypes = [i32, i32, P, P, P, P, i32, i32, i32, P, P, P, P]
        lib.oracle_checking_stage.restype = None
        lib.oracle_checking_stage.argtypes = [i32, i32, P, i32, i32, i32, P, P, P, P, i64]
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _csr(row_ptr, col, val):
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    return row_ptr, col, val


def spmv(row_ptr, col, val, x) -> np.ndarray:
    """Plain FP64 row loop (Sec. 2.1), one thread."""
    row_ptr, col, val = _csr(row_ptr, col, val)
    x = np.ascontiguousarray(x, dtype=np.float64)
    m = len(row_ptr) - 1
    y = np.empty(m, dtype=np.float64)
    _load().oracle_spmv_rowloop(m, _p(row_ptr), _p(col), _p(val), _p(x), _p(y))
    return y


def spmv_omp(row_ptr, col, val, x, nthreads: int = 0, y=None):
    """Row loop with rows split over OpenMP threads (the paper's CPU row-block
    method, Sec. 4.3).  Returns (y, threads used)."""
    row_ptr, col, val = _csr(row_ptr, col, val)
    x = np.ascontiguousarray(x, dtype=np.float64)
    m = len(row_ptr) - 1
    if y is None:
        y = np.empty(m, dtype=np.float64)
    used = _load().oracle_spmv_rowloop_omp(m, _p(row_ptr), _p(col), _p(val), _p(x), _p(y),
                                           nthreads)
    return y, used


def spmv_range(row_ptr, col, val, x, B: int, E: int) -> np.ndarray:
    """The row loop over the nonzeros [B, E) only (Sec. 2.1 restricted to one
    shard of a product split by entry ranges)."""
    row_ptr, col, val = _csr(row_ptr, col, val)
    x = np.ascontiguousarray(x, dtype=np.float64)
    m = len(row_ptr) - 1
    y = np.empty(m, dtype=np.float64)
    _load().oracle_spmv_range(m, _p(row_ptr), _p(col), _p(val), _p(x), int(B), int(E), _p(y))
    return y


def spmv_dot2(row_ptr, col, val, x):
    """Compensated reference y (Dot2) and per-row scale sum_k |val_k x[col_k]|."""
    row_ptr, col, val = _csr(row_ptr, col, val)
    x = np.ascontiguousarray(x, dtype=np.float64)
    m = len(row_ptr) - 1
    y = np.empty(m, dtype=np.float64)
    s = np.empty(m, dtype=np.float64)
    _load().oracle_spmv_dot2(m, _p(row_ptr), _p(col), _p(val), _p(x), _p(y), _p(s))
    return y, s


def num_tiles(nnz: int, L: int) -> int:
    return (nnz + L - 1) // L


def tile_offsets(row_ptr, L: int) -> np.ndarray:
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    m = len(row_ptr) - 1
    nnz = int(row_ptr[-1]) if m >= 0 else 0
    out = np.empty(num_tiles(nnz, L) + 1, dtype=np.int32)
    _load().oracle_tile_offsets(m, nnz, _p(row_ptr), L, _p(out))
    return out


def descriptors(row_ptr, L: int, tile_offset=None) -> np.ndarray:
    """Raw descriptor words, shape (ntiles, ceil(L/32)), uint32."""
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    m = len(row_ptr) - 1
    nnz = int(row_ptr[-1])
    if tile_offset is None:
        tile_offset = tile_offsets(row_ptr, L)
    nt = num_tiles(nnz, L)
    wpt = (L + 31) // 32
    out = np.empty((nt, wpt), dtype=np.uint32)
    _load().oracle_descriptors(m, nnz, _p(row_ptr), L, _p(tile_offset), _p(out))
    return out


def tile_flags(row_ptr, L: int, tile_offset=None):
    """(dirty uint8[ntiles], nseg int32[ntiles])."""
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    m = len(row_ptr) - 1
    nnz = int(row_ptr[-1])
    if tile_offset is None:
        tile_offset = tile_offsets(row_ptr, L)
    nt = num_tiles(nnz, L)
    dirty = np.empty(nt, dtype=np.uint8)
    nseg = np.empty(nt, dtype=np.int32)
    _load().oracle_tile_flags(m, nnz, _p(row_ptr), L, _p(tile_offset), _p(dirty), _p(nseg))
    return dirty, nseg


def bunch_count(nnz: int, T: int, W: int, S: int) -> int:
    L = T * W
    return (nnz + S * L - 1) // (S * L)


def speculative_stage(row_ptr, col, val, x, T: int, W: int, S: int):
    """Algorithm 1 simulated.  Returns dict with y (speculative), sync_idx,
    sync_val, speculator (dirty tile ids in bunch order), dirty_counter."""
    row_ptr, col, val = _csr(row_ptr, col, val)
    x = np.ascontiguousarray(x, dtype=np.float64)
    m = len(row_ptr) - 1
    nnz = int(row_ptr[-1])
    nb = bunch_count(nnz, T, W, S)
    y = np.empty(m, dtype=np.float64)
    sync_idx = np.full(max(nb, 1), -1, dtype=np.int32)
    sync_val = np.zeros(max(nb, 1), dtype=np.float64)
    spec = np.full(max(num_tiles(nnz, T * W), 1), -1, dtype=np.int32)
    dc = _load().oracle_speculative_stage(m, nnz, _p(row_ptr), _p(col), _p(val), _p(x),
                                          T, W, S, _p(y), _p(sync_idx), _p(sync_val), _p(spec))
    if dc < 0:
        raise MemoryError("oracle_speculative_stage")
    return dict(y=y, sync_idx=sync_idx[:nb], sync_val=sync_val[:nb],
                speculator=spec[:dc], dirty_counter=int(dc))


def checking_stage(row_ptr, T: int, W: int, S: int, st: dict) -> np.ndarray:
    """Synchronisation + re-arrangement (Sec. 3.2) applied to a copy of the
    speculative y from ``speculative_stage``; returns the final y."""
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    m = len(row_ptr) - 1
    nnz = int(row_ptr[-1])
    y = st["y"].copy()
    si = np.ascontiguousarray(st["sync_idx"], dtype=np.int32)
    sv = np.ascontiguousarray(st["sync_val"], dtype=np.float64)
    sp = np.ascontiguousarray(st["speculator"], dtype=np.int32)
    _load().oracle_checking_stage(m, nnz, _p(row_ptr), T, W, S, _p(y), _p(si), _p(sv), _p(sp),
                                  st["dirty_counter"])
    return y
