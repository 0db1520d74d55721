"""Torch-facing convenience layer over the C ABI: device allocations (CSR
arrays, y, workspace) are torch tensors; every computation is a call into
libssspmv.so through ``ssspmv``."""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

import torch

from . import ssspmv as _c


@dataclass
class DeviceCSR:
    m: int
    n: int
    nnz: int
    row_ptr: torch.Tensor  # int32 [m+1]
    col: torch.Tensor      # int32 [nnz], 16-byte aligned
    val: torch.Tensor      # f64 [nnz], 16-byte aligned


def to_device(row_ptr, col, val, n: int, device="cuda") -> DeviceCSR:
    """Copy host CSR arrays (numpy or torch) to fresh device tensors."""
    rp = torch.as_tensor(row_ptr, dtype=torch.int32).to(device).contiguous()
    c = torch.as_tensor(col, dtype=torch.int32).to(device).contiguous()
    v = torch.as_tensor(val, dtype=torch.float64).to(device).contiguous()
    m = rp.numel() - 1
    return DeviceCSR(m, int(n), int(c.numel()), rp, c, v)


def workspace_for(A: DeviceCSR, opts=None, device="cuda") -> torch.Tensor:
    nbytes = _c.ssspmv_workspace_bytes(A.m, A.nnz, 8, opts)
    if nbytes <= 0:
        raise _c.SsspmvError(_c.SSSPMV_EINVAL, "ssspmv_workspace_bytes")
    return torch.empty(nbytes, dtype=torch.uint8, device=device)


def spmv_f64(A: DeviceCSR, x: torch.Tensor, y: torch.Tensor | None = None, opts=None,
             workspace: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """y = A x (FP64) on the device through ssspmv_csr_f64."""
    if y is None:
        y = torch.empty(A.m, dtype=torch.float64, device=x.device)
    if workspace is None:
        workspace = workspace_for(A, opts, device=x.device)
    rc = _c.ssspmv_csr_f64(A.m, A.n, A.nnz, A.row_ptr, A.col, A.val, x, y, opts=opts,
                           workspace=workspace, stream=stream)
    _c.check(rc, "ssspmv_csr_f64")
    return y


def spmv_f64_debug(A: DeviceCSR, x: torch.Tensor, opts=None, stream=None) -> dict:
    """Runs the product and returns y with the exported index artefacts
    (host numpy arrays) and the speculative y before calibration."""
    shape = _c.ssspmv_plan_shape(A.m, A.nnz, 8, opts)
    dev = x.device
    nt, nb, W = shape["ntiles"], shape["nbunches"], shape["W"]
    y = torch.full((A.m,), float("nan"), dtype=torch.float64, device=dev)
    y_spec = torch.empty(A.m, dtype=torch.float64, device=dev)
    toff = torch.empty(nt + 1, dtype=torch.int32, device=dev)
    desc = torch.zeros(max(nt * W, 1), dtype=torch.int32, device=dev)
    info = torch.zeros(max(nt, 1), dtype=torch.int32, device=dev)
    sidx = torch.zeros(max(nb, 1), dtype=torch.int32, device=dev)
    ws = workspace_for(A, opts, device=dev)
    rc = _c.ssspmv_csr_f64_debug(A.m, A.n, A.nnz, A.row_ptr, A.col, A.val, x, y, opts=opts,
                                 workspace=ws, stream=stream, tile_offset=toff, desc=desc,
                                 tile_info=info, sync_idx=sidx, y_spec=y_spec)
    _c.check(rc, "ssspmv_csr_f64_debug")
    return dict(y=y.cpu().numpy(), y_spec=y_spec.cpu().numpy(),
                tile_offset=toff.cpu().numpy(),
                desc=desc.cpu().numpy().view("uint32")[: nt * W].reshape(nt, W),
                tile_info=info.cpu().numpy().view("uint32")[:nt],
                sync_idx=sidx.cpu().numpy()[:nb], shape=shape)


# ---------------------------------------------------------------------------
# one product split by tile ranges (ssspmv_csr_f64_range)

def split_tiles(ntiles: int, shards: int) -> list:
    """Contiguous tile ranges [t0, t1) of nearly equal length, one per shard."""
    return [(ntiles * g // shards, ntiles * (g + 1) // shards) for g in range(shards)]


def spmv_f64_shard(A: DeviceCSR, x: torch.Tensor, y: torch.Tensor, t0: int, t1: int, opts=None,
                   stream=None) -> np.ndarray:
    """This shard's rows of y = A x (tiles [t0, t1)) written into y, and its
    seam record as six floats (row0, row1, status, 0, partial0, partial1)."""
    r_first, r_last = _c.ssspmv_range_bounds(A.m, A.nnz, A.row_ptr, t0, t1, opts, stream)
    nbytes = _c.ssspmv_range_workspace_bytes(A.m, A.nnz, t0, t1, r_first, r_last, opts)
    if nbytes <= 0:
        raise _c.SsspmvError(_c.SSSPMV_EINVAL, "ssspmv_range_workspace_bytes")
    ws = torch.empty(nbytes, dtype=torch.uint8, device=x.device)
    seam = torch.zeros(_c.SEAM_BYTES, dtype=torch.uint8, device=x.device)
    _c.check(_c.ssspmv_csr_f64_range(A.m, A.n, A.nnz, A.row_ptr, A.col, A.val, x, y, t0, t1,
                                     r_first, r_last, seam, opts=opts, workspace=ws,
                                     stream=stream), "ssspmv_csr_f64_range")
    s = _c.seams_from_bytes(seam.cpu().numpy().tobytes())[0]
    return np.array([s.row[0], s.row[1], s.status, 0, s.val[0], s.val[1]], dtype=np.float64)


def merge_seams(records) -> tuple:
    """Rows cut at shard ends and their final values from the shards' seam
    records (six floats each, in shard order), through ssspmv_seam_merge."""
    arr = (_c.ssspmv_seam * len(records))()
    for d, r in zip(arr, records):
        d.row[0], d.row[1], d.status = int(r[0]), int(r[1]), int(r[2])
        d.val[0], d.val[1] = float(r[4]), float(r[5])
    return _c.ssspmv_seam_merge(arr)
