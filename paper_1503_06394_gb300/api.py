"""Convenience layer over the C ABI: keeps the CSR arrays and the workspace as
torch CUDA tensors and forwards to libcld.  No arithmetic of the estimator is
done here."""
from __future__ import annotations

import numpy as np

from . import _binding as B

_DTYPES = {"f32": B.CLD_F32, "bf16": B.CLD_BF16, "f64": B.CLD_F64}
_KINDS = {"spd": B.CLD_SPD, "general": B.CLD_GENERAL}


def _torch():
    import torch

    if not torch.cuda.is_available():
        raise RuntimeError("a CUDA device is required (libcld has no CPU path)")
    return torch


def _values_tensor(torch, val, dtype, device):
    if isinstance(val, np.ndarray):
        if dtype == "bf16":
            if val.dtype != np.uint16:
                raise TypeError("bf16 values must be given as uint16 bit patterns or a torch.bfloat16 tensor")
            return torch.from_numpy(val.view(np.int16)).to(device).view(torch.bfloat16)
        return torch.from_numpy(np.ascontiguousarray(val, dtype=np.float32 if dtype == "f32" else np.float64)).to(device)
    want = {"f32": torch.float32, "bf16": torch.bfloat16, "f64": torch.float64}[dtype]
    if val.dtype != want:
        raise TypeError("values tensor must be %s for dtype %s" % (want, dtype))
    return val.to(device).contiguous()


class CsrLogdet:
    """A CSR matrix on the GPU bound to a libcld handle.

    rowptr (d+1, int64), col (nnz, int32), val (nnz; f32 / bf16 / f64) may be
    numpy arrays or torch tensors; they are copied to ``device`` once and kept
    alive for the handle's lifetime.  ``kind='general'`` estimates log|det C|
    through C^T C (Algorithm 2)."""

    def __init__(self, rowptr, col, val, dtype: str = "f32", kind: str = "spd", device="cuda", stream=None):
        torch = _torch()
        self.torch = torch
        self.device = torch.device(device)
        self.rowptr = torch.as_tensor(np.asarray(rowptr, dtype=np.int64) if isinstance(rowptr, np.ndarray) else rowptr,
                                      dtype=torch.int64).to(self.device).contiguous()
        self.col = torch.as_tensor(np.asarray(col, dtype=np.int32) if isinstance(col, np.ndarray) else col,
                                   dtype=torch.int32).to(self.device).contiguous()
        self.val = _values_tensor(torch, val, dtype, self.device)
        self.d = int(self.rowptr.numel() - 1)
        self.nnz = int(self.col.numel())
        self.dtype = dtype
        self.kind = kind
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.h = B.cld_create_csr(self.d, self.nnz, self.rowptr, self.col, self.val, _DTYPES[dtype],
                                  _KINDS[kind], self.stream.cuda_stream)
        self.ws = None
        self.ws_bytes = 0

    # -- workspace ---------------------------------------------------------
    def reserve(self, n: int, M: int, with_grad: int = 0):
        need = B.cld_workspace_size(self.h, n, M, with_grad)
        if self.ws is None or self.ws_bytes < need:
            self.ws = None
            self.ws = self.torch.empty(need, dtype=self.torch.uint8, device=self.device)
            self.ws_bytes = need
            B.cld_set_workspace(self.h, self.ws, need)
        return need

    # -- interval ----------------------------------------------------------
    def set_interval(self, a: float, b: float):
        B.cld_set_interval(self.h, float(a), float(b))

    def auto_interval(self, lanczos_iters: int = 0):
        self.reserve(0, 1)
        return B.cld_auto_interval(self.h, lanczos_iters)

    # -- estimate ----------------------------------------------------------
    def estimate(self, n: int, M: int, seed: int = 0, moments: bool = False, details: bool = False,
                 raise_on_spectrum: bool = True):
        self.reserve(n, M)
        g, se, t, st = B.cld_estimate(self.h, n, M, seed, moments=moments, raise_on_spectrum=raise_on_spectrum)
        out = {"logdet": g, "stderr": se, "status": st}
        if moments:
            out["t"] = t
        if details and st == B.CLD_OK:
            out["c"], out["gamma_p"] = B.cld_last_details(self.h, n, M)
        return out

    def grad(self, n: int, M: int, seed: int = 0):
        """(logdet, dGamma/dval as an FP32 CUDA tensor of nnz entries); the
        interval is held fixed.  Needs a structurally symmetric pattern."""
        self.reserve(n, M, 1)
        G = self.torch.empty(self.nnz, dtype=self.torch.float32, device=self.device)
        g = B.cld_grad(self.h, n, M, seed, G)
        return g, G

    def set_grad_checkpoint(self, interval: int):
        """0: grad() keeps every w_j; K >= 2: keeps checkpoint pairs every K
        steps and recomputes segments (about 2n/K + K blocks)."""
        B.cld_set_grad_checkpoint(self.h, interval)

    def set_kernel_variant(self, variant: int):
        B.cld_set_kernel_variant(self.h, variant)

    def set_graph(self, on: bool = True):
        B.cld_set_graph(self.h, on)

    def autotune(self, n: int, M: int, reps: int = 8):
        """Picks the fastest recurrence-step variant for this matrix (n, M
        size the workspace)."""
        self.reserve(n, M)
        return B.cld_autotune(self.h, M, reps)

    def set_profiling(self, on: bool = True):
        B.cld_set_profiling(self.h, on)

    def last_timing(self):
        return B.cld_last_timing(self.h)

    def launch_config(self, M: int):
        return B.cld_launch_config(self.h, M)

    def close(self):
        if getattr(self, "h", None):
            B.cld_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class DenseLogdet(CsrLogdet):
    """A dense d x d SPD matrix (BF16, row-major, leading dimension ld) on the
    tensor-core path.  ``matrix``: a torch.bfloat16 CUDA tensor of shape
    (d, ld) or (d, d), or a numpy uint16 array of BF16 bit patterns."""

    def __init__(self, matrix, d=None, device="cuda", stream=None):
        torch = _torch()
        self.torch = torch
        self.device = torch.device(device)
        if isinstance(matrix, np.ndarray):
            if matrix.dtype != np.uint16:
                raise TypeError("numpy input must be uint16 BF16 bit patterns")
            t = torch.from_numpy(matrix.view(np.int16)).to(self.device).view(torch.bfloat16)
        else:
            if matrix.dtype != torch.bfloat16:
                raise TypeError("dense matrix must be torch.bfloat16")
            t = matrix.to(self.device)
        rows, cols = t.shape
        self.d = int(d if d is not None else rows)
        ld = (cols + 7) // 8 * 8
        if ld != cols or not t.is_contiguous():
            pad = torch.zeros((rows, ld), dtype=torch.bfloat16, device=self.device)
            pad[:, :cols] = t
            t = pad
        self.val = t
        self.ld = ld
        self.nnz = 0
        self.dtype = "bf16"
        self.kind = "spd"
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.h = B.cld_create_dense(self.d, ld, self.val, B.CLD_BF16, B.CLD_SPD, self.stream.cuda_stream)
        self.ws = None
        self.ws_bytes = 0


class CsrBatchLogdet(CsrLogdet):
    """Many matrices in one block-diagonal CSR (global indices); block b holds
    rows [blk_rows[b], blk_rows[b+1]).  estimate() returns per-block arrays."""

    def __init__(self, blk_rows, rowptr, col, val, dtype: str = "f32", kind: str = "spd", device="cuda",
                 stream=None):
        torch = _torch()
        self.torch = torch
        self.device = torch.device(device)
        self.blk_rows = np.ascontiguousarray(blk_rows, dtype=np.int64)
        self.nb = int(self.blk_rows.shape[0] - 1)
        self.rowptr = torch.as_tensor(np.asarray(rowptr, dtype=np.int64) if isinstance(rowptr, np.ndarray) else rowptr,
                                      dtype=torch.int64).to(self.device).contiguous()
        self.col = torch.as_tensor(np.asarray(col, dtype=np.int32) if isinstance(col, np.ndarray) else col,
                                   dtype=torch.int32).to(self.device).contiguous()
        self.val = _values_tensor(torch, val, dtype, self.device)
        self.d = int(self.rowptr.numel() - 1)
        self.nnz = int(self.col.numel())
        self.dtype = dtype
        self.kind = kind
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.h = B.cld_create_batch(self.blk_rows, self.nnz, self.rowptr, self.col, self.val, _DTYPES[dtype],
                                    _KINDS[kind], self.stream.cuda_stream)
        self.ws = None
        self.ws_bytes = 0

    def set_intervals(self, a, b):
        B.cld_batch_set_intervals(self.h, a, b)

    def auto_intervals(self):
        self.reserve(0, 1)
        return B.cld_batch_auto_intervals(self.h, self.nb)

    def set_tile_rows(self, rows: int):
        B.cld_batch_set_tile_rows(self.h, rows)

    @property
    def tile_rows(self) -> int:
        """Rows per work tile (chosen by autotune(), or set_tile_rows())."""
        return B.cld_batch_get_tile_rows(self.h)

    def estimate(self, n: int, M: int, seed: int = 0):
        self.reserve(n, M)
        g, se = B.cld_batch_estimate(self.h, self.nb, n, M, seed)
        return {"logdet": g, "stderr": se}


def logdet(rowptr, col, val, n: int, M: int, seed: int = 0, interval=None, dtype: str = "f32",
           kind: str = "spd", lanczos_iters: int = 0):
    """One-call estimate: returns (logdet, stderr).  ``interval=None`` computes
    [a, b] on the device (Gershgorin / norm bounds, optional Lanczos)."""
    m = CsrLogdet(rowptr, col, val, dtype=dtype, kind=kind)
    try:
        if interval is None:
            m.auto_interval(lanczos_iters)
        else:
            m.set_interval(*interval)
        r = m.estimate(n, M, seed)
        return r["logdet"], r["stderr"]
    finally:
        m.close()


def logdet_host(rowptr, col, val, a: float, b: float, n: int, M: int, seed: int = 0, dtype: str = "f32",
                kind: str = "spd", workspace=None, stream=None):
    """Estimate from host arrays through ``cld_logdet_csr_host`` (the library
    copies them to the device itself).  ``workspace``: optional preallocated
    uint8 CUDA tensor of at least ``cld_host_workspace_size`` bytes."""
    torch = _torch()
    d = int(len(rowptr) - 1)
    nnz = int(len(col))
    need = B.cld_host_workspace_size(d, nnz, _DTYPES[dtype], n, M)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device="cuda")
    s = stream if stream is not None else torch.cuda.current_stream()
    return B.cld_logdet_csr_host(d, nnz, rowptr, col, val, _DTYPES[dtype], _KINDS[kind], float(a), float(b),
                                 n, M, seed, workspace, need, s.cuda_stream)
