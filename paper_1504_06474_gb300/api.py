"""Torch-facing convenience layer over the C ABI: device allocations (CSR
arrays, y, workspace) are torch tensors; every computation is a call into
libssspmv.so through ``ssspmv``."""
from __future__ import annotations

from dataclasses import dataclass

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
