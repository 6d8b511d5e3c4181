"""Oracle for the phi-combination method (arXiv 2509.26475): ctypes wrapper of phicomb_oracle.c.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package.  The library in ``paper_2509_26475_gb300`` never
does, and the two share no code.

Functions follow the paper:
  * :func:`select`     -- Algorithm 1 (scaling s and shift xi*), Section 3.
  * :func:`solve`      -- Algorithm 3 (w_i = sum_j alpha_i^j phi_j(t_i A) v_j, i = 1..r), Section 4.
  * :func:`solve_single` -- Algorithm 2 (one combination), Section 4.
  * :func:`objective_at` -- the objective f(xi) of Algorithm 1 at given shifts.
  * :func:`unit_vector`  -- the splitmix64 unit-vector draw used when Algorithm 1 gets no v.

Parity status: every function is pinned by tests under ``tests/`` (closed forms, brute-force
augmented exponentials, invariants) except the exact location of xi*, which is "parity unpinned":
the objective has a rounding-noise floor near its minimum, so only f(xi*) and s are pinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "phicomb_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, INVALID_ARG, NONFINITE, TERM_CAP = 0, 1, 2, 3
FLAG_NO_V0 = 1
MAX_M = 256


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, -ffp-contract=off, OpenMP over sparse-product rows)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("rowptr", ctypes.c_void_p), ("colidx", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class _SelectOut(ctypes.Structure):
    _fields_ = [("xi", ctypes.c_double), ("s", ctypes.c_double), ("s0", ctypes.c_double),
                ("f_star", ctypes.c_double), ("r", ctypes.c_int32), ("evals", ctypes.c_int32),
                ("L", ctypes.c_double * (MAX_M + 1))]


class _Stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("s_int", ctypes.c_int32), ("series_terms", ctypes.c_int32),
                ("max_inner_terms", ctypes.c_int32), ("recovery_terms", ctypes.c_int64),
                ("spmm_count", ctypes.c_int64)]


_FN = ctypes.CFUNCTYPE(ctypes.c_double, ctypes.c_void_p, ctypes.c_double)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            lib.orc_select.argtypes = [ctypes.POINTER(_Csr), ctypes.c_int, ctypes.c_double, ctypes.c_double, P,
                                       ctypes.c_uint64, ctypes.c_int, P, ctypes.POINTER(_SelectOut)]
            lib.orc_select.restype = ctypes.c_int
            lib.orc_objective_at.argtypes = [ctypes.POINTER(_Csr), ctypes.c_int, ctypes.c_double, P, P,
                                             ctypes.c_int, P, ctypes.POINTER(ctypes.c_double),
                                             ctypes.POINTER(ctypes.c_int)]
            lib.orc_objective_at.restype = ctypes.c_int
            lib.orc_solve.argtypes = [ctypes.POINTER(_Csr), ctypes.c_int, ctypes.c_int, P, P, P, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_uint, ctypes.c_int, P,
                                      ctypes.POINTER(_Stats)]
            lib.orc_solve.restype = ctypes.c_int
            lib.orc_solve_single.argtypes = [ctypes.POINTER(_Csr), ctypes.c_int, P, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int, P,
                                             ctypes.POINTER(_Stats)]
            lib.orc_solve_single.restype = ctypes.c_int
            lib.orc_unit_vector.argtypes = [ctypes.c_int64, ctypes.c_uint64, P]
            lib.orc_unit_vector.restype = None
            lib.orc_minimize.argtypes = [_FN, P, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]
            lib.orc_minimize.restype = ctypes.c_double
            lib.orc_set_threads.argtypes = [ctypes.c_int]
            lib.orc_set_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def set_threads(nthreads: int) -> int:
    """Set the OpenMP thread count of the sparse products (0 = leave); returns the count in use."""
    return int(_load().orc_set_threads(int(nthreads)))


def _csr(A):
    rowptr = np.ascontiguousarray(A.rowptr, dtype=np.int32)
    colidx = np.ascontiguousarray(A.colidx, dtype=np.int32)
    val = np.ascontiguousarray(A.values, dtype=np.float64)
    c = _Csr(int(A.n), int(colidx.size), rowptr.ctypes.data, colidx.ctypes.data, val.ctypes.data)
    return c, (rowptr, colidx, val)


def _ptr(a):
    return None if a is None else a.ctypes.data


def unit_vector(n: int, seed: int) -> np.ndarray:
    """Components 2u-1, u = splitmix64(seed, i) >> 11 scaled by 2^-53 (not normalised)."""
    v = np.empty(int(n), dtype=np.float64)
    _load().orc_unit_vector(int(n), ctypes.c_uint64(int(seed) & (2**64 - 1)), v.ctypes.data)
    return v


def select(A, m: int = 61, tol: float = 2.0**-53, delta: float = 0.8, v=None, seed: int = 0x5EED,
           max_evals: int = 200, return_basis: bool = False):
    """Algorithm 1: returns dict(xi, s, s0, f_star, r, evals, L[0..r]) (and the basis V, n x (m+1))."""
    lib = _load()
    c, keep = _csr(A)
    vv = None if v is None else np.ascontiguousarray(v, dtype=np.float64)
    V = np.empty((m + 1, int(A.n)), dtype=np.float64)
    out = _SelectOut()
    st = lib.orc_select(ctypes.byref(c), int(m), float(tol), float(delta), _ptr(vv),
                        ctypes.c_uint64(int(seed) & (2**64 - 1)), int(max_evals), V.ctypes.data, ctypes.byref(out))
    if st != OK:
        raise RuntimeError(f"oracle select failed with status {st}")
    res = dict(xi=out.xi, s=out.s, s0=out.s0, f_star=out.f_star, r=int(out.r), evals=int(out.evals),
               L=np.array(out.L[: out.r + 1]))
    if return_basis:
        res["V"] = V
    return res


def objective_at(A, xis, m: int = 61, delta: float = 0.8, v=None, seed: int = 0x5EED):
    """f(xi) of Algorithm 1 for each xi in ``xis`` (same basis construction as :func:`select`)."""
    lib = _load()
    c, keep = _csr(A)
    vv = unit_vector(A.n, seed) if v is None else np.ascontiguousarray(v, dtype=np.float64)
    x = np.ascontiguousarray(np.atleast_1d(xis), dtype=np.float64)
    f = np.empty_like(x)
    s0 = ctypes.c_double(0.0)
    r = ctypes.c_int(0)
    st = lib.orc_objective_at(ctypes.byref(c), int(m), float(delta), vv.ctypes.data, x.ctypes.data, int(x.size),
                              f.ctypes.data, ctypes.byref(s0), ctypes.byref(r))
    if st != OK:
        raise RuntimeError(f"oracle objective failed with status {st}")
    return f, s0.value, r.value


def solve(A, V, t, alpha, tol: float, s: float, xi: float, flags: int = 0, max_terms: int = 0,
          check: bool = True):
    """Algorithm 3.  V is (p+1, n) with v_j in row j; returns (W (r, n), stats dict)."""
    lib = _load()
    c, keep = _csr(A)
    Vc = np.ascontiguousarray(V, dtype=np.float64)
    p = Vc.shape[0] - 1
    t = np.ascontiguousarray(np.atleast_1d(t), dtype=np.float64)
    alpha = np.ascontiguousarray(np.atleast_1d(alpha), dtype=np.float64)
    r = t.size
    if alpha.size != r:
        raise ValueError("t and alpha must have the same length")
    W = np.empty((r, int(A.n)), dtype=np.float64)
    st = _Stats()
    rc = lib.orc_solve(ctypes.byref(c), int(p), int(r), Vc.ctypes.data, t.ctypes.data, alpha.ctypes.data,
                       float(tol), float(s), float(xi), int(flags), int(max_terms), W.ctypes.data, ctypes.byref(st))
    stats = dict(status=st.status, s_int=st.s_int, series_terms=st.series_terms,
                 max_inner_terms=st.max_inner_terms, recovery_terms=st.recovery_terms, spmm_count=st.spmm_count)
    if check and rc != OK:
        raise RuntimeError(f"oracle solve failed with status {rc}")
    return W, stats


def solve_single(A, V, t: float, alpha: float, tol: float, s: float, xi: float, max_terms: int = 0):
    """Algorithm 2 (one combination).  Returns (w (n,), stats dict)."""
    lib = _load()
    c, keep = _csr(A)
    Vc = np.ascontiguousarray(V, dtype=np.float64)
    p = Vc.shape[0] - 1
    w = np.empty(int(A.n), dtype=np.float64)
    st = _Stats()
    rc = lib.orc_solve_single(ctypes.byref(c), int(p), Vc.ctypes.data, float(t), float(alpha), float(tol), float(s),
                              float(xi), int(max_terms), w.ctypes.data, ctypes.byref(st))
    if rc != OK:
        raise RuntimeError(f"oracle solve_single failed with status {rc}")
    return w, dict(status=st.status, s_int=st.s_int, series_terms=st.series_terms,
                   max_inner_terms=st.max_inner_terms, recovery_terms=st.recovery_terms, spmm_count=st.spmm_count)


def minimize(fn, a: float, b: float, tabs: float, max_evals: int = 200):
    """The oracle's Brent minimiser applied to a Python function: returns (x, f(x), evaluations)."""
    lib = _load()
    cb = _FN(lambda ctx, x: float(fn(x)))
    fmin = ctypes.c_double(0.0)
    ne = ctypes.c_int(0)
    x = lib.orc_minimize(cb, None, float(a), float(b), float(tabs), int(max_evals), ctypes.byref(fmin), ctypes.byref(ne))
    return x, fmin.value, ne.value
