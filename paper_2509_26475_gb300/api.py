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
                recovery_terms=s.recovery_terms, spmm_count=s.spmm_count, xi=s.xi, s=s.s,
                op_format=("csr", "ell", "dia", "lowrank", "function")[s.op_format] if 0 <= s.op_format <= 4 else s.op_format,
                op_slots=s.op_slots)


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
    lowrank = isinstance(A, DeviceLowRank)
    fnop = isinstance(A, FunctionOperator)
    if lowrank:
        out_sz = ctypes.c_size_t(0)
        capi.check(lib.phic_lowrank_select_workspace_size(A.n, A.k, int(m), ctypes.byref(out_sz)),
                   "phic_lowrank_select_workspace_size")
        nbytes = int(out_sz.value)
    elif fnop:
        out_sz = ctypes.c_size_t(0)
        capi.check(lib.phic_fn_select_workspace_size(A.n, int(m), ctypes.byref(out_sz)), "phic_fn_select_workspace_size")
        nbytes = int(out_sz.value)
    else:
        nbytes = select_workspace_bytes(A.n, m)
    ws = workspace if workspace is not None else workspaces.get("select", nbytes, dev)
    vptr = None
    if v is not None:
        if v.dtype != torch.float64 or not v.is_cuda or not v.is_contiguous() or v.numel() != A.n:
            raise ValueError("v must be a contiguous CUDA float64 tensor with n entries")
        vptr = v.data_ptr()
    c = A.struct()
    fn = lib.phic_lowrank_select_params if lowrank else lib.phic_fn_select_params if fnop else lib.phic_select_params
    st = fn(ctypes.byref(c), ctypes.byref(opts), vptr, ws.data_ptr(), ws.numel(), params.data_ptr(),
            _stream_handle(stream))
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
    lowrank = isinstance(A, DeviceLowRank)
    fnop = isinstance(A, FunctionOperator)
    if lowrank:
        out_sz = ctypes.c_size_t(0)
        capi.check(lib.phic_lowrank_solve_workspace_size(A.n, A.k, int(p), int(r), int(prec), ctypes.byref(out_sz)),
                   "phic_lowrank_solve_workspace_size")
        nbytes = int(out_sz.value)
    elif fnop:
        out_sz = ctypes.c_size_t(0)
        capi.check(lib.phic_fn_solve_workspace_size(A.n, int(p), int(r), int(prec), ctypes.byref(out_sz)),
                   "phic_fn_solve_workspace_size")
        nbytes = int(out_sz.value)
    else:
        nbytes = solve_workspace_bytes(A.n, A.nnz, p, r, prec)
    ws = workspace if workspace is not None else workspaces.get(("fn" if fnop else "solve", prec), nbytes, dev)
    c = A.struct()
    fn = lib.phic_lowrank_solve if lowrank else lib.phic_fn_solve if fnop else lib.phic_solve
    st = fn(ctypes.byref(c), int(p), int(r), V.data_ptr(), t.ctypes.data, alpha.ctypes.data, float(tol),
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


# ---- batched launches ------------------------------------------------------------------------------
@dataclass
class BatchItem:
    """One instance of a batch.  ``V`` is (p+1, n) (p rows with ``no_v0``) in the precision of A's
    values; ``params``, ``W`` and ``stats`` are allocated when not given.  ``select`` runs Algorithm 1
    for the instance at the start of its team's work; ``s_hint`` (host) only steers the planner."""

    A: DeviceCSR
    V: torch.Tensor | None
    t: tuple
    alpha: tuple
    tol: float = 2.0**-53
    select: bool = True
    solve: bool = True
    no_v0: bool = False
    s_hint: float = 0.0
    max_terms: int = 0
    params: torch.Tensor | None = None
    W: torch.Tensor | None = None
    stats: torch.Tensor | None = None
    v_select: torch.Tensor | None = None

    def prepare(self):
        dev = self.A.rowptr.device
        dt = _TORCH_DT[self.A.prec]
        t = np.atleast_1d(np.asarray(self.t, dtype=np.float64))
        if self.params is None:
            self.params = new_params(dev)
        if self.solve:
            if self.V is None or self.V.dtype != dt or not self.V.is_cuda or not self.V.is_contiguous() or \
                    self.V.dim() != 2 or self.V.shape[1] != self.A.n:
                raise ValueError(f"V must be a contiguous CUDA {dt} tensor of shape (p+1, n)")
            if self.W is None:
                self.W = torch.empty((t.size, self.A.n), dtype=dt, device=dev)
            if self.stats is None:
                self.stats = new_stats(dev)
        return self

    @property
    def p(self) -> int:
        if self.V is None:
            return 0
        return self.V.shape[0] if self.no_v0 else self.V.shape[0] - 1

    def struct(self) -> capi.phic_batch_item:
        t = np.atleast_1d(np.asarray(self.t, dtype=np.float64))
        a = np.atleast_1d(np.asarray(self.alpha, dtype=np.float64))
        if t.size != a.size or not 1 <= t.size <= capi.PHIC_MAX_R:
            raise ValueError("t and alpha must have the same length, at most PHIC_MAX_R")
        it = capi.phic_batch_item()
        it.A = self.A.struct()
        it.p, it.r = self.p, int(t.size)
        it.flags = (capi.PHIC_NO_V0 if self.no_v0 else 0) | (capi.PHIC_BATCH_SELECT if self.select else 0) | \
            (0 if self.solve else capi.PHIC_BATCH_NO_SOLVE)
        it.max_terms = int(self.max_terms)
        it.V = self.V.data_ptr() if self.V is not None else None
        it.W = self.W.data_ptr() if self.W is not None else None
        it.params = self.params.data_ptr()
        it.stats = self.stats.data_ptr() if self.stats is not None else None
        it.v_select = self.v_select.data_ptr() if self.v_select is not None else None
        it.tol, it.s_hint = float(self.tol), float(self.s_hint)
        for i in range(t.size):
            it.t[i], it.alpha[i] = float(t[i]), float(a[i])
        return it


def _select_opts(m=61, delta=0.8, seed=0x5EED, max_evals=200):
    opts = capi.phic_select_opts()
    capi.load().phic_select_opts_default(ctypes.byref(opts))
    opts.m, opts.delta, opts.seed, opts.max_evals = int(m), float(delta), int(seed) & (2**64 - 1), int(max_evals)
    return opts


def _item_array(items):
    arr = (capi.phic_batch_item * len(items))()
    for i, it in enumerate(items):
        arr[i] = it.prepare().struct()
    return arr


def _config(cfg):
    if cfg is None:
        return None
    if isinstance(cfg, capi.phic_batch_config):
        return cfg
    return capi.phic_batch_config(int(cfg.get("rows_per_cta", 0)), int(cfg.get("blocks_per_sm", 0)),
                                  int(cfg.get("max_steps", 0)), 0)


def batch_workspace_bytes(items, select_opts=None) -> int:
    arr = _item_array(items)
    out = ctypes.c_size_t(0)
    opts = select_opts or _select_opts()
    capi.check(capi.load().phic_batch_workspace_size(arr, len(items), ctypes.byref(opts), ctypes.byref(out)),
               "phic_batch_workspace_size")
    return int(out.value)


class Batch:
    """Many independent instances in one persistent cooperative launch (``phic_batch_*``).

        b = Batch([BatchItem(A1, V1, t1, a1), BatchItem(A2, V2, t2, a2, tol=2**-24), ...])
        b.launch()                 # one kernel launch for every instance (capturable in a CUDA graph)
        W1 = b.items[0].W

    ``config`` is a dict with ``rows_per_cta``, ``blocks_per_sm`` and ``max_steps`` (see
    phic_batch_config) or None for the defaults; ``autotune`` picks one by timing the batch."""

    def __init__(self, items, config=None, select_opts=None, workspace: torch.Tensor | None = None, stream=None):
        self.lib = capi.load()
        self.items = list(items)
        self.arr = _item_array(self.items)
        self.opts = select_opts or _select_opts()
        nbytes = batch_workspace_bytes(self.items, self.opts)
        dev = self.items[0].A.rowptr.device
        self.ws = workspace if workspace is not None and workspace.numel() >= nbytes else \
            torch.empty(max(nbytes, 256), dtype=torch.uint8, device=dev)
        self.cfg = _config(config)
        h = ctypes.c_void_p(0)
        st = self.lib.phic_batch_create(self.arr, len(self.items), ctypes.byref(self.opts),
                                        ctypes.byref(self.cfg) if self.cfg is not None else None,
                                        self.ws.data_ptr(), self.ws.numel(), _stream_handle(stream), ctypes.byref(h))
        capi.check(st, "phic_batch_create")
        self.handle = h
        self._pending = torch.zeros(1, dtype=torch.int32, device=dev)

    def launch(self, stream=None):
        capi.check(self.lib.phic_batch_launch(self.handle, _stream_handle(stream)), "phic_batch_launch")

    def resume(self, stream=None):
        capi.check(self.lib.phic_batch_resume(self.handle, _stream_handle(stream)), "phic_batch_resume")

    def pending(self, stream=None) -> int:
        capi.check(self.lib.phic_batch_pending(self.handle, self._pending.data_ptr(), _stream_handle(stream)),
                   "phic_batch_pending")
        return int(self._pending.item())

    def info(self) -> dict:
        inf = capi.phic_batch_info()
        capi.check(self.lib.phic_batch_info_get(self.handle, ctypes.byref(inf)), "phic_batch_info_get")
        return {k: getattr(inf, k) for k, _ in capi.phic_batch_info._fields_}

    def stats(self) -> list:
        return [read_stats(it.stats) if it.stats is not None else None for it in self.items]

    def params(self) -> list:
        return [read_params(it.params) for it in self.items]

    def close(self):
        if getattr(self, "handle", None):
            self.lib.phic_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune(items, candidates=None, reps: int = 3, select_opts=None, workspace: torch.Tensor | None = None,
             stream=None):
    """Times the batch under each candidate configuration (dicts as for Batch) and returns
    (best config dict, its median ms).  None searches the library's default grid."""
    lib = capi.load()
    items = list(items)
    arr = _item_array(items)
    opts = select_opts or _select_opts()
    nbytes = batch_workspace_bytes(items, opts)
    dev = items[0].A.rowptr.device
    ws = workspace if workspace is not None and workspace.numel() >= nbytes else \
        torch.empty(max(nbytes, 256), dtype=torch.uint8, device=dev)
    cand = None
    ncand = 0
    if candidates:
        cand = (capi.phic_batch_config * len(candidates))(*[_config(c) for c in candidates])
        ncand = len(candidates)
    best = capi.phic_batch_config()
    ms = ctypes.c_double(0.0)
    st = lib.phic_batch_autotune(arr, len(items), ctypes.byref(opts), ws.data_ptr(), ws.numel(), cand, ncand,
                                 int(reps), _stream_handle(stream), ctypes.byref(best), ctypes.byref(ms))
    capi.check(st, "phic_batch_autotune")
    return {"rows_per_cta": best.rows_per_cta, "blocks_per_sm": best.blocks_per_sm, "max_steps": best.max_steps}, \
        float(ms.value)


# ---- serving loop ----------------------------------------------------------------------------------
def _info_dict(info: capi.phic_request_info) -> dict:
    p, s = info.params, info.stats
    return dict(state=info.state, status=info.status, submit_ns=info.submit_ns, admit_ns=info.admit_ns,
                done_ns=info.done_ns, slices=info.slices,
                params=dict(xi=p.xi, s=p.s, s0=p.s0, f_star=p.f_star, r=p.r, evals=p.evals, status=p.status),
                stats=dict(status=s.status, s_int=s.s_int, series_terms=s.series_terms,
                           max_inner_terms=s.max_inner_terms, recovery_terms=s.recovery_terms,
                           spmm_count=s.spmm_count, xi=s.xi, s=s.s))


def _host(a, dtype, pin):
    x = torch.as_tensor(np.ascontiguousarray(a)).to(dtype)
    return x.pin_memory() if pin else x.contiguous()


class HostOperator:
    """Host-side (page-locked) CSR arrays of an operator to register with a Server."""

    def __init__(self, A, prec: str = "f64", pin: bool = True):
        dt = torch.float32 if prec in ("f32", capi.PHIC_F32, torch.float32) else torch.float64
        self.rowptr = _host(A.rowptr, torch.int32, pin)
        self.colidx = _host(A.colidx, torch.int32, pin)
        self.values = _host(A.values, dt, pin)
        self.n, self.nnz, self.prec = int(A.n), int(self.colidx.numel()), prec_of(dt)

    def struct(self) -> capi.phic_operator:
        return capi.phic_operator(self.n, self.nnz, self.rowptr.data_ptr(), self.colidx.data_ptr(),
                                  self.values.data_ptr(), self.prec, 0)


class HostRequest:
    """Host-side (page-locked) buffers of one request: the CSR operator (or a registered operator's id),
    V and the result W."""

    def __init__(self, A, V, t, alpha, tol: float = 2.0**-53, prec: str = "f64", no_v0: bool = False,
                 max_terms: int = 0, pin: bool = True, op: int = 0):
        dt = torch.float32 if prec in ("f32", capi.PHIC_F32, torch.float32) else torch.float64
        self.op = int(op)
        if self.op:
            self.rowptr = self.colidx = self.values = None
            n, nnz = int(A), 0
        else:
            self.rowptr = _host(A.rowptr, torch.int32, pin)
            self.colidx = _host(A.colidx, torch.int32, pin)
            self.values = _host(A.values, dt, pin)
            n, nnz = int(A.n), int(self.colidx.numel())
        self.V = _host(V, dt, pin)
        self.t = np.atleast_1d(np.asarray(t, dtype=np.float64))
        self.alpha = np.atleast_1d(np.asarray(alpha, dtype=np.float64))
        self.n, self.nnz = n, nnz
        self.prec = prec_of(dt)
        self.no_v0 = bool(no_v0)
        self.p = self.V.shape[0] if no_v0 else self.V.shape[0] - 1
        self.r = int(self.t.size)
        self.W = torch.empty((self.r, self.n), dtype=dt, pin_memory=pin)
        self.tol = float(tol)
        self.max_terms = int(max_terms)

    def struct(self) -> capi.phic_request:
        q = capi.phic_request()
        q.n, q.nnz = self.n, self.nnz
        if not self.op:
            q.rowptr, q.colidx, q.values = self.rowptr.data_ptr(), self.colidx.data_ptr(), self.values.data_ptr()
        q.op = self.op
        q.V, q.W = self.V.data_ptr(), self.W.data_ptr()
        q.prec, q.p, q.r = self.prec, self.p, self.r
        q.flags = capi.PHIC_NO_V0 if self.no_v0 else 0
        q.tol, q.max_terms = self.tol, self.max_terms
        for i in range(self.r):
            q.t[i], q.alpha[i] = float(self.t[i]), float(self.alpha[i])
        return q


class Server:
    """Continuous-batching request loop (phic_server_*): a worker thread in the library admits requests
    by device memory and runs them together in batched slices.

        srv = Server(arena_bytes=8 << 30)
        rid = srv.submit(HostRequest(A, V, t, alpha))
        info = srv.wait(rid); W = srv.result(rid)
    """

    def __init__(self, arena_bytes: int = 4 << 30, rows_per_cta: int = 0, blocks_per_sm: int = 0,
                 max_steps: int = 0, max_active: int = 0, device: int = 0, m: int = 0, slice_us: float = 0.0):
        self.lib = capi.load()
        self.arena = torch.empty(int(arena_bytes), dtype=torch.uint8, device=f"cuda:{device}")
        cfg = capi.phic_server_config(self.arena.data_ptr(), self.arena.numel(), int(rows_per_cta), int(blocks_per_sm),
                                      int(max_steps), int(max_active), int(device), int(m), float(slice_us))
        h = ctypes.c_void_p(0)
        capi.check(self.lib.phic_server_create(ctypes.byref(cfg), ctypes.byref(h)), "phic_server_create")
        self.handle = h
        self.requests = {}

    def submit(self, req: HostRequest) -> int:
        rid = ctypes.c_int64(0)
        q = req.struct()
        capi.check(self.lib.phic_server_submit(self.handle, ctypes.byref(q), ctypes.byref(rid)), "phic_server_submit")
        self.requests[rid.value] = req
        return int(rid.value)

    def add_operator(self, op: HostOperator) -> int:
        oid = ctypes.c_int64(0)
        capi.check(self.lib.phic_server_add_operator(self.handle, ctypes.byref(op.struct()), ctypes.byref(oid)),
                   "phic_server_add_operator")
        self.requests[oid.value] = op
        return int(oid.value)

    def operator_params(self, oid: int):
        ready = ctypes.c_int32(0)
        prm = capi.phic_params()
        capi.check(self.lib.phic_server_operator_params(self.handle, int(oid), ctypes.byref(ready), ctypes.byref(prm)),
                   "phic_server_operator_params")
        if not ready.value:
            return None
        return dict(xi=prm.xi, s=prm.s, s0=prm.s0, f_star=prm.f_star, r=prm.r, evals=prm.evals, status=prm.status)

    def remove_operator(self, oid: int):
        capi.check(self.lib.phic_server_remove_operator(self.handle, int(oid)), "phic_server_remove_operator")

    def query(self, rid: int) -> dict:
        info = capi.phic_request_info()
        capi.check(self.lib.phic_server_query(self.handle, int(rid), ctypes.byref(info)), "phic_server_query")
        return _info_dict(info)

    def wait(self, rid: int, timeout_ms: float = -1.0) -> dict:
        info = capi.phic_request_info()
        capi.check(self.lib.phic_server_wait(self.handle, int(rid), float(timeout_ms), ctypes.byref(info)),
                   "phic_server_wait")
        return _info_dict(info)

    def result(self, rid: int) -> torch.Tensor:
        return self.requests[rid].W

    def counters(self) -> dict:
        c = capi.phic_server_counters()
        capi.check(self.lib.phic_server_counters_get(self.handle, ctypes.byref(c)), "phic_server_counters_get")
        return {k: getattr(c, k) for k, _ in capi.phic_server_counters._fields_}

    def close(self):
        if getattr(self, "handle", None):
            self.lib.phic_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- matrix-free low-rank operators -----------------------------------------------------------------
@dataclass
class DeviceLowRank:
    """A = U W^T with U, W (n, k) contiguous CUDA tensors of one precision (k <= PHIC_MAX_RANK),
    applied matrix-free; accepted by select_params and solve in place of a DeviceCSR."""

    U: torch.Tensor
    W: torch.Tensor

    @property
    def n(self) -> int:
        return int(self.U.shape[0])

    @property
    def k(self) -> int:
        return int(self.U.shape[1])

    @property
    def prec(self) -> int:
        return prec_of(self.U.dtype)

    @property
    def nnz(self) -> int:
        return 0

    def struct(self) -> capi.phic_lowrank:
        for x in (self.U, self.W):
            if not x.is_cuda or not x.is_contiguous() or x.dim() != 2:
                raise ValueError("U and W must be contiguous (n, k) CUDA tensors")
        if self.U.shape != self.W.shape or self.U.dtype != self.W.dtype:
            raise ValueError("U and W must have the same shape and dtype")
        return capi.phic_lowrank(self.n, self.k, self.prec, self.U.data_ptr(), self.W.data_ptr())

    @property
    def rowptr(self):  # device of the operator, for the helpers that allocate next to it
        return self.U


class FunctionOperator:
    """An operator given by its product Y = A X (the phic_fn_* entry points): accepted by select_params and
    solve in place of a DeviceCSR.  ``apply`` is either a C function pointer of type phic_apply_fn (an int,
    e.g. ``ctypes.cast(lib.phic_csr_apply, c_void_p).value``, with ``ctx`` its context pointer) or a Python
    callable ``apply(X, Y, w, prec, stream)`` that receives X (n, ldx) and Y (n, ldy) as CUDA tensor views
    over the library's buffers (their first w columns are the block) and a torch stream, and enqueues
    Y[:, :w] = A X[:, :w] on that stream without allocating or synchronising (solve calls it while the
    library captures a CUDA graph).  ``norm_bound`` bounds ||A||_inf from above."""

    def __init__(self, n: int, apply, norm_bound: float, dtype=torch.float64, ctx: int | None = None):
        self.n = int(n)
        self.dtype = dtype
        self.norm_bound = float(norm_bound)
        self._keep = []
        if callable(apply) and not isinstance(apply, int):
            user = apply

            def trampoline(_ctx, X, ldx, Y, ldy, w, prec, stream):
                try:
                    dt = _TORCH_DT[int(prec)]
                    Xt = _device_view(X, self.n, int(ldx), dt)
                    Yt = _device_view(Y, self.n, int(ldy), dt)
                    s = torch.cuda.ExternalStream(int(stream)) if stream else torch.cuda.current_stream()
                    with torch.cuda.stream(s):
                        user(Xt, Yt, int(w), int(prec), s)
                    return 0
                except Exception:  # the library reports a failed product as PHIC_CUDA_ERROR
                    import traceback

                    traceback.print_exc()
                    return 1

            cfn = capi.APPLY_FN(trampoline)
            self._keep.append(cfn)
            self._fnptr = ctypes.cast(cfn, ctypes.c_void_p).value
            self._ctx = None
        else:
            self._fnptr = int(apply)
            self._ctx = ctx

    @classmethod
    def from_csr(cls, A: "DeviceCSR") -> "FunctionOperator":
        """The library's own CSR product as the function (phic_csr_apply); the bound is ||A||_inf."""
        lib = capi.load()
        csr = A.struct()
        vals = A.values.double() if A.values.dtype != torch.float64 else A.values
        rows = torch.repeat_interleave(torch.arange(A.n, device=vals.device), A.rowptr[1:] - A.rowptr[:-1])
        bound = float(torch.zeros(A.n, dtype=torch.float64, device=vals.device).index_add_(0, rows, vals.abs()).max())
        op = cls(A.n, ctypes.cast(lib.phic_csr_apply, ctypes.c_void_p).value, bound, A.values.dtype,
                 ctypes.addressof(csr))
        op._keep += [csr, A]
        return op

    @property
    def prec(self) -> int:
        return prec_of(self.dtype)

    @property
    def nnz(self) -> int:
        return 0

    @property
    def rowptr(self):  # the device the operator lives on, as DeviceCSR exposes it
        return torch.empty(0, device="cuda")

    def struct(self) -> capi.phic_fn_op:
        c = capi.phic_fn_op(self.n, self.prec, 0, self._fnptr, self._ctx, self.norm_bound)
        self._keep.append(c)
        return c


class _CudaArray:
    """A CUDA array interface over a raw device pointer (no copy), for torch.as_tensor."""

    def __init__(self, ptr: int, shape, strides_bytes, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (int(ptr), False),
                                         "strides": tuple(strides_bytes), "version": 3}


def _device_view(ptr: int, n: int, ld: int, dtype) -> torch.Tensor:
    es = 8 if dtype == torch.float64 else 4
    typestr = "<f8" if dtype == torch.float64 else "<f4"
    return torch.as_tensor(_CudaArray(ptr, (n, ld), (ld * es, es), typestr), device="cuda")
