"""ctypes binding of libssspmv.so (include/ssspmv.h): the same entry points
under the same names, with argument marshalling only.  Every step of the
product runs in the library's CUDA kernels; there is no Python or CPU
fallback, and loading fails loudly when the library has not been built.

Array arguments may be torch tensors (device memory, contiguous) or raw
integer addresses.  Streams may be torch.cuda.Stream objects, raw handles or
None (the current torch stream when torch is importable, else the legacy
default stream).
"""
from __future__ import annotations

import ctypes
import os
import re

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libssspmv.so")
HEADER_PATH = os.path.join(os.path.dirname(_PKG), "include", "ssspmv.h")

SSSPMV_OK = 0
SSSPMV_EINVAL = -1
SSSPMV_EWORKSPACE = -2
SSSPMV_ECUDA = -3
SSSPMV_EDEVICE = -4
SSSPMV_EUNSUPPORTED = -5
SSSPMV_ETOOLARGE = -6
SSSPMV_NOALLOC_SCRATCH_BYTES = 8 << 20
SSSPMV_MAX_DIM = 2147483647 - 256
SSSPMV_DEV_TIMEOUT, SSSPMV_DEV_RANGE, SSSPMV_DEV_CALIB, SSSPMV_DEV_BATCH = 1, 2, 4, 8


class SsspmvError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = _lib().ssspmv_strerror(code).decode()
        if code == SSSPMV_ECUDA:
            msg += " (cudaError %d)" % _lib().ssspmv_last_cuda_error()
        super().__init__("%s: %s (%d)" % (where, msg, code))


class ssspmv_opts(ctypes.Structure):
    _fields_ = [("W", ctypes.c_int32), ("S", ctypes.c_int32), ("block_warps", ctypes.c_int32),
                ("variant", ctypes.c_int32), ("timer", ctypes.c_void_p)]


_L = None
P = ctypes.c_void_p
i32, i64, u32, sz = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_size_t
OPTS = ctypes.POINTER(ssspmv_opts)

_SIGS = {
    "ssspmv_plan_shape": (ctypes.c_int, [i32, i32, i32, OPTS, P, P, P, P, P]),
    "ssspmv_workspace_bytes": (sz, [i32, i32, i32, OPTS]),
    "ssspmv_csr_f64": (ctypes.c_int, [i32, i32, i32, P, P, P, P, P, OPTS, P, sz, P]),
    "ssspmv_csr_f32": (ctypes.c_int, [i32, i32, i32, P, P, P, P, P, OPTS, P, sz, P]),
    "ssspmv_csr_bf16f32": (ctypes.c_int, [i32, i32, i32, P, P, P, P, P, OPTS, P, sz, P]),
    "ssspmv_csr_f64_noalloc": (ctypes.c_int, [i32, i32, i32, P, P, P, P, P, OPTS, P]),
    "ssspmv_host_buffer_bytes": (sz, [i32, i32, i32, OPTS]),
    "ssspmv_csr_f64_host": (ctypes.c_int, [i32, i32, i32, P, P, P, P, P, OPTS, P, sz, P]),
    "ssspmv_csr_f64_debug": (ctypes.c_int, [i32, i32, i32, P, P, P, P, P, OPTS, P, sz, P,
                                            P, P, P, P, P]),
    "ssspmv_validate_csr": (ctypes.c_int, [i32, i32, i32, P, P, P, P]),
    "ssspmv_device_status": (ctypes.c_int, [P, sz, P, ctypes.c_int, P]),
    "ssspmv_supported_w": (ctypes.c_int, [P, i32, P]),
    "ssspmv_timer_create": (ctypes.c_int, [i32, P]),
    "ssspmv_timer_destroy": (None, [P]),
    "ssspmv_timer_reset": (None, [P]),
    "ssspmv_timer_read": (ctypes.c_int, [P, P, i32, P]),
    "ssspmv_cached_workspace": (ctypes.c_int, [P, P, P]),
    "ssspmv_release_workspaces": (None, []),
    "ssspmv_plan_create": (ctypes.c_int, [i32, i32, i32, P, i32, OPTS, P, sz, P, P]),
    "ssspmv_plan_execute": (ctypes.c_int, [P, P, P, P, P, P, P]),
    "ssspmv_plan_workspace": (ctypes.c_int, [P, P, P]),
    "ssspmv_plan_destroy": (None, [P]),
    "ssspmv_csr_f64_axpby": (ctypes.c_int, [i32, i32, i32, P, P, P, P, P, ctypes.c_double,
                                            ctypes.c_double, OPTS, P, sz, P]),
    "ssspmv_plan_execute_axpby": (ctypes.c_int, [P, P, P, P, P, ctypes.c_double,
                                                 ctypes.c_double, P, P]),
    "ssspmv_batched_workspace_bytes": (sz, [i32, i64, i32, OPTS]),
    "ssspmv_features_scratch_bytes": (sz, []),
    "ssspmv_features": (ctypes.c_int, [i32, i32, i32, P, P, P, P]),
    "ssspmv_mlp_param_count": (i64, [i32, i32, i32, i32]),
    "ssspmv_mlp_scratch_floats": (sz, [i32, i32, i32, i32, i32]),
    "ssspmv_mlp_forward": (ctypes.c_int, [P, P, i32, i32, i32, i32, i32, P, P, P]),
    "ssspmv_mlp_backward": (ctypes.c_int, [P, P, P, i32, i32, i32, i32, i32, P, P, P, P]),
    "ssspmv_mlp_adam": (ctypes.c_int, [P, P, P, P, i64, ctypes.c_float, ctypes.c_float,
                                       ctypes.c_float, ctypes.c_float, ctypes.c_float, i32, P]),
    "ssspmv_mlp_select": (ctypes.c_int, [P, P, i32, i32, i32, i32, i32, P, P, P]),
    "ssspmv_csr_batched_f32": (ctypes.c_int, [i32, P, i64, OPTS, P, sz, P]),
    "ssspmv_range_bounds": (ctypes.c_int, [i32, i32, P, OPTS, i64, i64, P, P, P]),
    "ssspmv_range_workspace_bytes": (sz, [i32, i32, i64, i64, i32, i32, OPTS]),
    "ssspmv_csr_f64_range": (ctypes.c_int, [i32, i32, i32, P, P, P, P, P, i64, i64, i32, i32, P,
                                            OPTS, P, sz, P]),
    "ssspmv_seam_merge": (ctypes.c_int, [i32, P, P, P, P]),
    "ssspmv_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "ssspmv_last_cuda_error": (ctypes.c_int, []),
    "ssspmv_version": (ctypes.c_int, []),
}


def _lib():
    global _L
    if _L is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libssspmv.so is not built (run __graft_entry__.build() or "
                              "python -m paper_1504_06474_gb300._build)")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _L = lib
    return _L


def declared_functions() -> list[str]:
    """Names of the functions include/ssspmv.h declares."""
    with open(HEADER_PATH) as f:
        text = re.sub(r"/\*.*?\*/", "", f.read(), flags=re.S)
    return sorted(set(re.findall(r"\b(ssspmv_[a-z0-9_]+)\s*\(", text)))


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if hasattr(a, "data_ptr"):
        if a.numel() and not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr() if a.numel() else None
    if hasattr(a, "ctypes"):  # numpy array (host)
        return a.ctypes.data if a.size else None
    raise TypeError("cannot take the address of %r" % type(a))


def _stream(s):
    if s is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


VARIANT_DEFAULT, VARIANT_SPECULATIVE, VARIANT_EXACT, VARIANT_ROWS = 0, 1, 2, 3


def make_opts(W: int = 0, S: int = 0, timer=None, variant: int = 0,
              block_warps: int = 0) -> ssspmv_opts:
    o = ssspmv_opts()
    o.W, o.S, o.block_warps, o.variant = W, S, block_warps, variant
    o.timer = timer
    return o


def _opts(o):
    return None if o is None else ctypes.byref(o)


def check(rc: int, where: str):
    if rc != SSSPMV_OK:
        raise SsspmvError(rc, where)


# --- entry points (same names as the C ABI) --------------------------------

def ssspmv_plan_shape(m, nnz, val_bytes=8, opts=None):
    W, L, S = i32(), i32(), i32()
    nt, nb = i64(), i64()
    rc = _lib().ssspmv_plan_shape(m, nnz, val_bytes, _opts(opts), ctypes.byref(W),
                                  ctypes.byref(L), ctypes.byref(S), ctypes.byref(nt),
                                  ctypes.byref(nb))
    check(rc, "ssspmv_plan_shape")
    return dict(W=W.value, L=L.value, S=S.value, ntiles=nt.value, nbunches=nb.value)


def ssspmv_workspace_bytes(m, nnz, val_bytes=8, opts=None) -> int:
    return int(_lib().ssspmv_workspace_bytes(m, nnz, val_bytes, _opts(opts)))


def ssspmv_csr_f64(m, n, nnz, row_ptr, col_idx, val, x, y, opts=None, workspace=None,
                   ws_bytes=None, stream=None) -> int:
    if ws_bytes is None:
        ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    return _lib().ssspmv_csr_f64(m, n, nnz, _ptr(row_ptr), _ptr(col_idx), _ptr(val), _ptr(x),
                                 _ptr(y), _opts(opts), _ptr(workspace), ws_bytes,
                                 _stream(stream))


def ssspmv_csr_f32(m, n, nnz, row_ptr, col_idx, val, x, y, opts=None, workspace=None,
                   ws_bytes=None, stream=None) -> int:
    if ws_bytes is None:
        ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    return _lib().ssspmv_csr_f32(m, n, nnz, _ptr(row_ptr), _ptr(col_idx), _ptr(val), _ptr(x),
                                 _ptr(y), _opts(opts), _ptr(workspace), ws_bytes,
                                 _stream(stream))


def ssspmv_csr_bf16f32(m, n, nnz, row_ptr, col_idx, val, x, y, opts=None, workspace=None,
                       ws_bytes=None, stream=None) -> int:
    if ws_bytes is None:
        ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    return _lib().ssspmv_csr_bf16f32(m, n, nnz, _ptr(row_ptr), _ptr(col_idx), _ptr(val),
                                     _ptr(x), _ptr(y), _opts(opts), _ptr(workspace), ws_bytes,
                                     _stream(stream))


def ssspmv_csr_f64_noalloc(m, n, nnz, row_ptr, col_idx, val, x, y, opts=None,
                           stream=None) -> int:
    """FP64 product with the library's fixed scratch instead of a workspace,
    for callers that cannot allocate device memory (see include/ssspmv.h)."""
    return _lib().ssspmv_csr_f64_noalloc(m, n, nnz, _ptr(row_ptr), _ptr(col_idx), _ptr(val),
                                         _ptr(x), _ptr(y), _opts(opts), _stream(stream))


def ssspmv_host_buffer_bytes(m, n, nnz, opts=None) -> int:
    return int(_lib().ssspmv_host_buffer_bytes(m, n, nnz, _opts(opts)))


def ssspmv_csr_f64_host(m, n, nnz, host_row_ptr, host_col_idx, host_val, host_x, host_y,
                        opts=None, dev_buffer=None, dev_bytes=None, stream=None) -> int:
    if dev_bytes is None:
        dev_bytes = dev_buffer.numel() * dev_buffer.element_size() if dev_buffer is not None else 0
    return _lib().ssspmv_csr_f64_host(m, n, nnz, _ptr(host_row_ptr), _ptr(host_col_idx),
                                      _ptr(host_val), _ptr(host_x), _ptr(host_y), _opts(opts),
                                      _ptr(dev_buffer), dev_bytes, _stream(stream))


def ssspmv_csr_f64_debug(m, n, nnz, row_ptr, col_idx, val, x, y, opts=None, workspace=None,
                         ws_bytes=None, stream=None, tile_offset=None, desc=None,
                         tile_info=None, sync_idx=None, y_spec=None) -> int:
    if ws_bytes is None:
        ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    return _lib().ssspmv_csr_f64_debug(m, n, nnz, _ptr(row_ptr), _ptr(col_idx), _ptr(val),
                                       _ptr(x), _ptr(y), _opts(opts), _ptr(workspace), ws_bytes,
                                       _stream(stream), _ptr(tile_offset), _ptr(desc),
                                       _ptr(tile_info), _ptr(sync_idx), _ptr(y_spec))


def ssspmv_validate_csr(m, n, nnz, row_ptr, col_idx, scratch, stream=None) -> int:
    return _lib().ssspmv_validate_csr(m, n, nnz, _ptr(row_ptr), _ptr(col_idx), _ptr(scratch),
                                      _stream(stream))


def ssspmv_device_status(workspace, ws_bytes=None, stream=None, clear=False) -> int:
    if ws_bytes is None:
        ws_bytes = workspace.numel() * workspace.element_size()
    bits = u32()
    rc = _lib().ssspmv_device_status(_ptr(workspace), ws_bytes, _stream(stream), int(clear),
                                     ctypes.byref(bits))
    check(rc, "ssspmv_device_status")
    return bits.value


def ssspmv_supported_w() -> list[int]:
    buf = (i32 * 16)()
    cnt = i32()
    _lib().ssspmv_supported_w(buf, 16, ctypes.byref(cnt))
    return [buf[i] for i in range(min(cnt.value, 16))]


def ssspmv_timer_create(capacity: int) -> int:
    h = ctypes.c_void_p()
    check(_lib().ssspmv_timer_create(capacity, ctypes.byref(h)), "ssspmv_timer_create")
    return h.value


def ssspmv_timer_destroy(timer: int) -> None:
    _lib().ssspmv_timer_destroy(timer)


def ssspmv_timer_reset(timer: int) -> None:
    _lib().ssspmv_timer_reset(timer)


def ssspmv_timer_read(timer: int, cap: int):
    """List of (partition, segsum, calibrate, whole call) times in ms."""
    buf = (ctypes.c_float * (4 * max(cap, 1)))()
    cnt = i32()
    check(_lib().ssspmv_timer_read(timer, buf, cap, ctypes.byref(cnt)), "ssspmv_timer_read")
    n = min(cnt.value, cap)
    return [tuple(buf[4 * i + j] for j in range(4)) for i in range(n)]


def ssspmv_cached_workspace(stream=None):
    """(pointer, bytes) of the library-owned workspace of this device and stream."""
    p, b = ctypes.c_void_p(), ctypes.c_size_t()
    rc = _lib().ssspmv_cached_workspace(_stream(stream), ctypes.byref(p), ctypes.byref(b))
    check(rc, "ssspmv_cached_workspace")
    return p.value, b.value


def ssspmv_release_workspaces() -> None:
    _lib().ssspmv_release_workspaces()


def ssspmv_plan_create(m, n, nnz, row_ptr, val_bytes=8, opts=None, workspace=None,
                       ws_bytes=None, stream=None) -> int:
    """Returns the plan handle (an int); raises SsspmvError on failure."""
    if ws_bytes is None:
        ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    h = ctypes.c_void_p()
    rc = _lib().ssspmv_plan_create(m, n, nnz, _ptr(row_ptr), val_bytes, _opts(opts),
                                   _ptr(workspace), ws_bytes, _stream(stream), ctypes.byref(h))
    check(rc, "ssspmv_plan_create")
    return h.value


def ssspmv_plan_execute(plan, col_idx, val, x, y, timer=None, stream=None) -> int:
    return _lib().ssspmv_plan_execute(plan, _ptr(col_idx), _ptr(val), _ptr(x), _ptr(y), timer,
                                      _stream(stream))


def ssspmv_plan_workspace(plan):
    p, b = ctypes.c_void_p(), ctypes.c_size_t()
    check(_lib().ssspmv_plan_workspace(plan, ctypes.byref(p), ctypes.byref(b)),
          "ssspmv_plan_workspace")
    return p.value, b.value


def ssspmv_csr_f64_axpby(m, n, nnz, row_ptr, col_idx, val, x, y, alpha, beta, opts=None,
                         workspace=None, ws_bytes=None, stream=None) -> int:
    if ws_bytes is None:
        ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    return _lib().ssspmv_csr_f64_axpby(m, n, nnz, _ptr(row_ptr), _ptr(col_idx), _ptr(val),
                                       _ptr(x), _ptr(y), alpha, beta, _opts(opts),
                                       _ptr(workspace), ws_bytes, _stream(stream))


def ssspmv_plan_execute_axpby(plan, col_idx, val, x, y, alpha, beta, timer=None,
                              stream=None) -> int:
    return _lib().ssspmv_plan_execute_axpby(plan, _ptr(col_idx), _ptr(val), _ptr(x), _ptr(y),
                                            alpha, beta, timer, _stream(stream))


def ssspmv_plan_destroy(plan) -> None:
    _lib().ssspmv_plan_destroy(plan)


class ssspmv_csr_desc(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("n", ctypes.c_int32), ("nnz", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("row_ptr", ctypes.c_void_p),
                ("col_idx", ctypes.c_void_p), ("val", ctypes.c_void_p), ("x", ctypes.c_void_p),
                ("y", ctypes.c_void_p)]


def batch_descriptors(mats) -> bytes:
    """Packs (m, n, nnz, row_ptr, col_idx, val, x, y) tuples (pointers or
    tensors) into the bytes of a descriptor array, to be copied to the device."""
    arr = (ssspmv_csr_desc * len(mats))()
    for d, (m, n, nnz, rp, col, val, x, y) in zip(arr, mats):
        d.m, d.n, d.nnz, d.reserved = m, n, nnz, 0
        d.row_ptr, d.col_idx, d.val, d.x, d.y = _ptr(rp), _ptr(col), _ptr(val), _ptr(x), _ptr(y)
    return bytes(arr)


def ssspmv_batched_workspace_bytes(count, total_nnz, val_bytes=4, opts=None) -> int:
    return int(_lib().ssspmv_batched_workspace_bytes(count, total_nnz, val_bytes, _opts(opts)))


def ssspmv_csr_batched_f32(count, mats, total_nnz, opts=None, workspace=None, ws_bytes=None,
                           stream=None) -> int:
    if ws_bytes is None:
        ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    return _lib().ssspmv_csr_batched_f32(count, _ptr(mats), total_nnz, _opts(opts),
                                         _ptr(workspace), ws_bytes, _stream(stream))


def ssspmv_features_scratch_bytes() -> int:
    return int(_lib().ssspmv_features_scratch_bytes())


def ssspmv_features(m, n, nnz, row_ptr, features, scratch, stream=None) -> int:
    return _lib().ssspmv_features(m, n, nnz, _ptr(row_ptr), _ptr(features), _ptr(scratch),
                                  _stream(stream))


def ssspmv_mlp_param_count(F, H1, H2, K) -> int:
    return int(_lib().ssspmv_mlp_param_count(F, H1, H2, K))


def ssspmv_mlp_scratch_floats(B, F, H1, H2, K) -> int:
    return int(_lib().ssspmv_mlp_scratch_floats(B, F, H1, H2, K))


def ssspmv_mlp_forward(params, X, B, F, H1, H2, K, scratch, out=None, stream=None) -> int:
    return _lib().ssspmv_mlp_forward(_ptr(params), _ptr(X), B, F, H1, H2, K, _ptr(scratch),
                                     _ptr(out), _stream(stream))


def ssspmv_mlp_backward(params, X, target, B, F, H1, H2, K, scratch, grad, loss=None,
                        stream=None) -> int:
    return _lib().ssspmv_mlp_backward(_ptr(params), _ptr(X), _ptr(target), B, F, H1, H2, K,
                                      _ptr(scratch), _ptr(grad), _ptr(loss), _stream(stream))


def ssspmv_mlp_adam(params, grad, m1, m2, n, lr, beta1=0.9, beta2=0.999, eps=1e-8,
                    weight_decay=0.0, step=1, stream=None) -> int:
    return _lib().ssspmv_mlp_adam(_ptr(params), _ptr(grad), _ptr(m1), _ptr(m2), n, lr, beta1,
                                  beta2, eps, weight_decay, step, _stream(stream))


def ssspmv_mlp_select(params, X, B, F, H1, H2, K, scratch, cls, stream=None) -> int:
    return _lib().ssspmv_mlp_select(_ptr(params), _ptr(X), B, F, H1, H2, K, _ptr(scratch),
                                    _ptr(cls), _stream(stream))


def ssspmv_strerror(code: int) -> str:
    return _lib().ssspmv_strerror(code).decode()


def ssspmv_last_cuda_error() -> int:
    return _lib().ssspmv_last_cuda_error()


def ssspmv_version() -> int:
    return _lib().ssspmv_version()


# --- tile-range shards and their seam records ------------------------------

class ssspmv_seam(ctypes.Structure):
    _fields_ = [("row", ctypes.c_int32 * 2), ("status", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("val", ctypes.c_double * 2)]


SEAM_BYTES = ctypes.sizeof(ssspmv_seam)


def ssspmv_range_bounds(m, nnz, row_ptr, t0, t1, opts=None, stream=None):
    """(r_first, r_last) of the tiles [t0, t1); synchronises the stream."""
    a, b = i32(), i32()
    check(_lib().ssspmv_range_bounds(m, nnz, _ptr(row_ptr), _opts(opts), t0, t1,
                                     ctypes.byref(a), ctypes.byref(b), _stream(stream)),
          "ssspmv_range_bounds")
    return a.value, b.value


def ssspmv_range_workspace_bytes(m, nnz, t0, t1, r_first, r_last, opts=None) -> int:
    return int(_lib().ssspmv_range_workspace_bytes(m, nnz, t0, t1, r_first, r_last,
                                                   _opts(opts)))


def ssspmv_csr_f64_range(m, n, nnz, row_ptr, col_idx, val, x, y, t0, t1, r_first, r_last, seam,
                         opts=None, workspace=None, ws_bytes=None, stream=None) -> int:
    """`seam` is a device buffer of SEAM_BYTES bytes (e.g. a uint8 tensor)."""
    if ws_bytes is None:
        ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    return _lib().ssspmv_csr_f64_range(m, n, nnz, _ptr(row_ptr), _ptr(col_idx), _ptr(val),
                                       _ptr(x), _ptr(y), t0, t1, r_first, r_last, _ptr(seam),
                                       _opts(opts), _ptr(workspace), ws_bytes, _stream(stream))


def seams_from_bytes(raw: bytes):
    """Host seam records from their raw bytes (one or more records)."""
    n = len(raw) // SEAM_BYTES
    arr = (ssspmv_seam * n).from_buffer_copy(raw[: n * SEAM_BYTES])
    return arr


def ssspmv_seam_merge(seams):
    """(rows, vals) of the cut rows from host seam records in shard order."""
    n = len(seams)
    arr = (ssspmv_seam * n)(*seams) if not isinstance(seams, ctypes.Array) else seams
    rows = (ctypes.c_int32 * (2 * max(n, 1)))()
    vals = (ctypes.c_double * (2 * max(n, 1)))()
    cnt = i32()
    check(_lib().ssspmv_seam_merge(n, arr, rows, vals, ctypes.byref(cnt)), "ssspmv_seam_merge")
    return list(rows[: cnt.value]), list(vals[: cnt.value])
