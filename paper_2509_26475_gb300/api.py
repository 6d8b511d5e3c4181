"""Python API over the C ABI: device memory and streams come from PyTorch, every step of the method
runs in libphicomb's CUDA kernels.

    A  = DeviceCSR.from_host(csr)                       # CSR operator in HBM (FP64 or FP32 values)
    P  = select_params(A)                               # Algorithm 1: xi*, s (stay on the device)
    W, st = solve(A, V, t, alpha, 2.0**-53, P)          # Algorithm 3: w_i, i = 1..r
    W = phimv(A, V, t, alpha)                           # both, with host or device inputs

All calls are asynchronous on the current (or given) CUDA stream.  ``check=True`` synchronises that
stream and raises :class:`~paper_2509_26475_gb300.capi.PhicError` when the device reports a status.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import capi

_TORCH_DT = {capi.PHIC_F64: torch.float64, capi.PHIC_F32: torch.float32}


def prec_of(dtype) -> int:
    if dtype in (torch.float64, np.float64, "f64", "float64"):
        return capi.PHIC_F64
    if dtype in (torch.float32, np.float32, "f32", "float32"):
        return capi.PHIC_F32
    raise ValueError(f"unsupported precision {dtype}")


def _stream_handle(stream) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


@dataclass
class DeviceCSR:
    """CSR operator resident on a CUDA device (int32 indices; FP64 or FP32 values)."""

    rowptr: torch.Tensor
    colidx: torch.Tensor
    values: torch.Tensor

    @property
    def n(self) -> int:
        return int(self.rowptr.numel() - 1)

    @property
    def nnz(self) -> int:
        return int(self.colidx.numel())

    @property
    def prec(self) -> int:
        return prec_of(self.values.dtype)

    @classmethod
    def from_host(cls, csr, device="cuda", dtype=torch.float64, non_blocking=False) -> "DeviceCSR":
        def t(a, dt):
            x = torch.as_tensor(np.ascontiguousarray(a)).to(dt)
            return x.to(device, non_blocking=non_blocking)

        return cls(t(csr.rowptr, torch.int32), t(csr.colidx, torch.int32), t(csr.values, dtype))

    def astype(self, dtype) -> "DeviceCSR":
        return DeviceCSR(self.rowptr, self.colidx, self.values.to(dtype))

    def struct(self) -> capi.phic_csr:
        for x in (self.rowptr, self.colidx, self.values):
            if not x.is_cuda or not x.is_contiguous():
                raise ValueError("DeviceCSR arrays must be contiguous CUDA tensors")
        return capi.phic_csr(self.n, self.nnz, self.rowptr.data_ptr(), self.colidx.data_ptr(),
                             self.values.data_ptr(), self.prec)


class _Workspaces:
    """Per-device scratch buffers reused across calls (grown on demand)."""

    def __init__(self):
        self._bufs = {}

    def get(self, key, nbytes: int, device) -> torch.Tensor:
        k = (key, str(device))
        buf = self._bufs.get(k)
        if buf is None or buf.numel() < nbytes:
            buf = torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)
            self._bufs[k] = buf
        return buf

    def clear(self):
        self._bufs.clear()


workspaces = _Workspaces()


def select_workspace_bytes(n: int, m: int = 61) -> int:
    out = ctypes.c_size_t(0)
    capi.check(capi.load().phic_select_workspace_size(int(n), int(m), ctypes.byref(out)), "phic_select_workspace_size")
    return int(out.value)


def solve_workspace_bytes(n: int, nnz: int, p: int, r: int, prec: int) -> int:
    out = ctypes.c_size_t(0)
    capi.check(capi.load().phic_solve_workspace_size(int(n), int(nnz), int(p), int(r), int(prec), ctypes.byref(out)),
               "phic_solve_workspace_size")
    return int(out.value)


def new_params(device="cuda") -> torch.Tensor:
    return torch.zeros(ctypes.sizeof(capi.phic_params), dtype=torch.uint8, device=device)


def new_stats(device="cuda") -> torch.Tensor:
    return torch.zeros(ctypes.sizeof(capi.phic_stats), dtype=torch.uint8, device=device)


def read_params(params: torch.Tensor) -> dict:
    raw = params.detach().cpu().numpy().tobytes()
    p = capi.phic_params.from_buffer_copy(raw)
    return dict(xi=p.xi, s=p.s, s0=p.s0, f_star=p.f_star, r=p.r, evals=p.evals, status=p.status)


def read_stats(stats: torch.Tensor) -> dict:
    raw = stats.detach().cpu().numpy().tobytes()
    s = capi.phic_stats.from_buffer_copy(raw)
    return dict(status=s.status, s_int=s.s_int, series_terms=s.series_terms, max_inner_terms=s.max_inner_terms,
                recovery_terms=s.recovery_terms, spmm_count=s.spmm_count, xi=s.xi, s=s.s)


def select_params(A: DeviceCSR, m: int = 61, tol: float = 2.0**-53, delta: float = 0.8, seed: int = 0x5EED,
                  max_evals: int = 200, v: torch.Tensor | None = None, out: torch.Tensor | None = None,
                  workspace: torch.Tensor | None = None, stream=None, check: bool = False) -> torch.Tensor:
    """Algorithm 1 (Section 3).  Returns the device phic_params buffer (xi*, s, diagnostics)."""
    lib = capi.load()
    dev = A.rowptr.device
    params = out if out is not None else new_params(dev)
    opts = capi.phic_select_opts()
    lib.phic_select_opts_default(ctypes.byref(opts))
    opts.m, opts.tol, opts.delta, opts.seed, opts.max_evals = int(m), float(tol), float(delta), int(seed) & (2**64 - 1), int(max_evals)
    nbytes = select_workspace_bytes(A.n, m)
    ws = workspace if workspace is not None else workspaces.get("select", nbytes, dev)
    vptr = None
    if v is not None:
        if v.dtype != torch.float64 or not v.is_cuda or not v.is_contiguous() or v.numel() != A.n:
            raise ValueError("v must be a contiguous CUDA float64 tensor with n entries")
        vptr = v.data_ptr()
    c = A.struct()
    st = lib.phic_select_params(ctypes.byref(c), ctypes.byref(opts), vptr, ws.data_ptr(), ws.numel(),
                                params.data_ptr(), _stream_handle(stream))
    capi.check(st, "phic_select_params")
    if check:
        (stream or torch.cuda.current_stream()).synchronize()
        info = read_params(params)
        capi.check(info["status"], "phic_select_params (device)")
    return params


def set_params(xi: float, s: float, out: torch.Tensor | None = None, device="cuda", stream=None) -> torch.Tensor:
    """Writes user-chosen (xi, s) into a device phic_params buffer."""
    params = out if out is not None else new_params(device)
    capi.check(capi.load().phic_params_set(params.data_ptr(), float(xi), float(s), _stream_handle(stream)),
               "phic_params_set")
    return params


def solve(A: DeviceCSR, V: torch.Tensor, t, alpha, tol: float, params: torch.Tensor, *, flags: int = 0,
          max_terms: int = 0, out: torch.Tensor | None = None, stats: torch.Tensor | None = None,
          workspace: torch.Tensor | None = None, stream=None, check: bool = False):
    """Algorithm 3 (Section 4).  V is a (p+1, n) CUDA tensor (p rows with ``PHIC_NO_V0``) in the
    precision of A's values; t and alpha are length-r host sequences.  Returns (W (r, n), stats)."""
    lib = capi.load()
    prec = A.prec
    dt = _TORCH_DT[prec]
    if V.dtype != dt or not V.is_cuda or not V.is_contiguous() or V.dim() != 2 or V.shape[1] != A.n:
        raise ValueError(f"V must be a contiguous CUDA {dt} tensor of shape (p+1, n)")
    p = V.shape[0] if (flags & capi.PHIC_NO_V0) else V.shape[0] - 1
    t = np.ascontiguousarray(np.atleast_1d(np.asarray(t, dtype=np.float64)))
    alpha = np.ascontiguousarray(np.atleast_1d(np.asarray(alpha, dtype=np.float64)))
    r = int(t.size)
    if alpha.size != r:
        raise ValueError("t and alpha must have the same length")
    dev = V.device
    W = out if out is not None else torch.empty((r, A.n), dtype=dt, device=dev)
    if W.shape != (r, A.n) or W.dtype != dt or not W.is_contiguous():
        raise ValueError("out has the wrong shape or dtype")
    stats = stats if stats is not None else new_stats(dev)
    nbytes = solve_workspace_bytes(A.n, A.nnz, p, r, prec)
    ws = workspace if workspace is not None else workspaces.get(("solve", prec), nbytes, dev)
    c = A.struct()
    st = lib.phic_solve(ctypes.byref(c), int(p), int(r), V.data_ptr(), t.ctypes.data, alpha.ctypes.data, float(tol),
                        params.data_ptr(), int(flags), int(max_terms), W.data_ptr(), ws.data_ptr(), ws.numel(),
                        stats.data_ptr(), int(prec), _stream_handle(stream))
    capi.check(st, "phic_solve")
    if check:
        (stream or torch.cuda.current_stream()).synchronize()
        capi.check(read_stats(stats)["status"], "phic_solve (device)")
    return W, stats


def phimv(A, V, t, alpha, tol: float = 2.0**-53, params: torch.Tensor | None = None, flags: int = 0,
          device="cuda", stream=None, check: bool = True):
    """w_i = sum_j alpha_i^j phi_j(t_i A) v_j, i = 1..r, end to end: ``A`` may be a host CSR (it is
    copied to the device) or a DeviceCSR; ``V`` may be a host array/tensor (copied in, result copied
    back) or a CUDA tensor (result stays on the device).  Algorithm 1 runs unless ``params`` is given."""
    host_io = not (isinstance(V, torch.Tensor) and V.is_cuda)
    if not isinstance(A, DeviceCSR):
        dt = torch.float32 if np.asarray(A.values).dtype == np.float32 else torch.float64
        A = DeviceCSR.from_host(A, device=device, dtype=dt, non_blocking=True)
    dt = _TORCH_DT[A.prec]
    if host_io:
        Vt = torch.as_tensor(np.ascontiguousarray(V) if not isinstance(V, torch.Tensor) else V).to(dt)
        Vd = Vt.to(device, non_blocking=True)
    else:
        Vd = V
    P = params if params is not None else select_params(A, stream=stream)
    W, st = solve(A, Vd, t, alpha, tol, P, flags=flags, stream=stream)
    if check:
        (stream or torch.cuda.current_stream()).synchronize()
        capi.check(read_params(P)["status"], "phic_select_params (device)")
        capi.check(read_stats(st)["status"], "phic_solve (device)")
    return W.cpu() if host_io else W
