"""CUDA path against the oracle, through the C ABI.

Algorithm 3 parity uses the same (s, xi) on both sides (Algorithm 1's minimiser is not bit-stable, see
test_gpu_select.py), fed to the device with phic_params_set.  Bars: relative 2-norm error per
combination <= 1e-12 at tol = 2^-53 (FP64) and <= 5e-6 at tol = 2^-24 (FP32 storage, against the FP64
oracle).  Sizes span several blocks of 256 rows with a ragged tail; the full-size workloads of the
benchmark are compared whole (the oracle runs them in seconds with OpenMP).
"""
import math

import numpy as np
import pytest
import torch

from paper_2509_26475_gb300 import api, capi
from paper_2509_26475_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL53, TOL24 = 2.0**-53, 2.0**-24


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2509_26475_gb300 import build

    build.build()
    capi.load()
    torch.cuda.set_device(0)


def _rel(W, ref):
    W = np.asarray(W, dtype=np.float64)
    return [float(np.linalg.norm(W[i] - ref[i]) / np.linalg.norm(ref[i])) for i in range(ref.shape[0])]


def _gpu_solve(Acsr, V, t, alpha, tol, s, xi, dtype=torch.float64, flags=0, max_terms=0):
    A = api.DeviceCSR.from_host(Acsr, dtype=dtype)
    Vd = torch.as_tensor(np.ascontiguousarray(V)).to(dtype).cuda()
    P = api.set_params(xi, s)
    W, st = api.solve(A, Vd, t, alpha, tol, P, flags=flags, max_terms=max_terms)
    torch.cuda.synchronize()
    return W.cpu().numpy(), api.read_stats(st)


def _check_parity(oracle_mod, Acsr, V, t, alpha, tol=TOL53, flags=0, bar=1e-12, s=None, xi=None):
    if s is None:
        sel = oracle_mod.select(Acsr)
        s, xi = sel["s"], sel["xi"]
    ref, ost = oracle_mod.solve(Acsr, V, t, alpha, TOL53 if tol < 1e-10 else tol, s, xi, flags=flags)
    W, gst = _gpu_solve(Acsr, V, t, alpha, tol, s, xi, flags=flags)
    assert gst["status"] == 0, gst
    errs = _rel(W, ref)
    assert max(errs) <= bar, errs
    assert gst["s_int"] == ost["s_int"]
    # term counts may differ by one only where a norm sits on the threshold
    assert abs(gst["series_terms"] - ost["series_terms"]) <= 1
    assert abs(gst["recovery_terms"] - ost["recovery_terms"]) <= max(1, ost["s_int"] // 10)
    return errs, gst, ost


def test_laplacian_32_full_path(oracle_mod):
    """The small benchmark case: 2-D Laplacian 32 x 32, p = 3, r = 1, t = 1e-3 (s_int = 1)."""
    w = wl.workload_laplacian_32()
    errs, gst, ost = _check_parity(oracle_mod, w["A"], w["V"], w["t"], w["alpha"])
    assert gst["series_terms"] == ost["series_terms"]


@pytest.mark.parametrize("nx,ny,p,r,tscale", [(40, 37, 3, 3, 3e-3), (23, 41, 2, 1, 1e-2), (64, 50, 4, 2, 6e-3),
                                              (17, 19, 5, 3, 2e-2)])
def test_convection_diffusion_recovery(oracle_mod, nx, ny, p, r, tscale):
    """Several blocks, ragged tails, s_int > 1 (recovery loop), distinct t_i and alpha_i."""
    h = 1.0 / (nx + 1)
    c = 1.0 / h**2
    b = 20.0 / h
    Acsr = wl._grid_operator((nx, ny), -4.0 * c - 2.0 * b, [c + b, c + b], [c, c])
    rng = np.random.default_rng(nx * 100 + ny)
    V = rng.standard_normal((p + 1, Acsr.n))
    t = tscale * np.array([1.0, 0.5, 0.3][:r])
    alpha = np.array([0.7, -1.2, 2.0][:r])
    errs, gst, ost = _check_parity(oracle_mod, Acsr, V, t, alpha)
    assert ost["s_int"] > 1


def test_nonnormal_dense_block(oracle_mod):
    rng = np.random.default_rng(3)
    n = 300
    Ad = np.triu(rng.standard_normal((n, n)), -3) * 2.0 + np.diag(np.linspace(-80, 3, n))
    Acsr = wl.dense_to_csr(Ad)
    V = rng.standard_normal((4, n))
    _check_parity(oracle_mod, Acsr, V, [0.05, 0.2, -0.1, 0.0], [1.0, 0.5, 2.0, -1.0])


@pytest.mark.parametrize("p,r", [(0, 1), (0, 3), (1, 2), (2, 1), (4, 3), (6, 5), (7, 16), (15, 8), (0, 5), (2, 2),
                                 (7, 3), (1, 5)])
def test_widths_and_padding(oracle_mod, p, r):
    """Block widths (p+1) r from 1 to 128, odd and padded layouts; widths 5, 6, 10, 24 and 35 take the
    series kernels with 3 or 5 columns a lane."""
    Acsr = wl.convection_diffusion(29, 2, 5.0)
    rng = np.random.default_rng(100 * p + r)
    V = rng.standard_normal((p + 1, Acsr.n))
    t = np.linspace(2e-3, 6e-3, r)
    alpha = np.linspace(0.5, 1.5, r)
    _check_parity(oracle_mod, Acsr, V, t, alpha)


def test_no_v0_flag(oracle_mod):
    Acsr = wl.convection_diffusion(31, 2, 3.0)
    rng = np.random.default_rng(9)
    V = rng.standard_normal((4, Acsr.n))
    sel = oracle_mod.select(Acsr)
    V0 = V.copy()
    V0[0] = 0.0
    ref, _ = oracle_mod.solve(Acsr, V0, [4e-3, 1e-3], [1.0, 0.5], TOL53, sel["s"], sel["xi"])
    W, st = _gpu_solve(Acsr, V[1:], [4e-3, 1e-3], [1.0, 0.5], TOL53, sel["s"], sel["xi"], flags=capi.PHIC_NO_V0)
    assert st["status"] == 0
    assert max(_rel(W, ref)) <= 1e-12


def test_fp32_storage_against_fp64_oracle(oracle_mod):
    Acsr = wl.convection_diffusion(60, 2, 50.0)
    rng = np.random.default_rng(5)
    V = rng.standard_normal((5, Acsr.n))
    t = np.array([0.25, 0.5, 0.75, 1.0]) * 2e-3
    alpha = np.ones(4)
    sel = oracle_mod.select(Acsr, tol=TOL24)
    ref, ost = oracle_mod.solve(Acsr, V, t, alpha, TOL53, sel["s"], sel["xi"])
    W, gst = _gpu_solve(Acsr, V, t, alpha, TOL24, sel["s"], sel["xi"], dtype=torch.float32)
    assert gst["status"] == 0
    assert max(_rel(W, ref)) <= 5e-6


def test_single_row_and_zero_time(oracle_mod):
    A1 = wl.diagonal([-3.5])
    V = np.array([[1.0], [0.5], [-2.0]])
    _check_parity(oracle_mod, A1, V, [0.7], [1.3])
    Acsr = wl.laplacian_2d(20)
    V = np.random.default_rng(2).standard_normal((3, Acsr.n))
    W, st = _gpu_solve(Acsr, V, [0.0], [2.0], TOL53, 100.0, -50.0)
    expect = V[0] + 2.0 * V[1] + 4.0 * V[2] / 2.0
    assert st["s_int"] == 1
    assert np.linalg.norm(W[0] - expect) / np.linalg.norm(expect) <= 1e-15


def test_empty_rows(oracle_mod):
    """Rows without nonzeros (A = 0 on part of the space): w = sum_j alpha^j v_j / j! there."""
    d = np.zeros(700)
    d[::3] = -np.linspace(1.0, 50.0, 234)
    full = wl.diagonal(d)
    keep = d != 0
    rowptr = np.concatenate([[0], np.cumsum(keep)]).astype(np.int32)
    Acsr = wl.CSR(700, rowptr, np.nonzero(keep)[0].astype(np.int32), d[keep])
    V = np.random.default_rng(4).standard_normal((3, 700))
    sel = oracle_mod.select(full)
    ref, _ = oracle_mod.solve(full, V, [0.1], [1.0], TOL53, sel["s"], sel["xi"])
    W, st = _gpu_solve(Acsr, V, [0.1], [1.0], TOL53, sel["s"], sel["xi"])
    assert st["status"] == 0 and max(_rel(W, ref)) <= 1e-12


def test_convdiff3d_64_full_size(oracle_mod):
    """The benchmark workload at full size (n = 262144, p = 3, r = 2, h = 1e-4 and 1e-2), compared whole."""
    oracle_mod.set_threads(0)
    for h in (1e-4, 1e-2):
        w = wl.workload_convdiff3d_64(h)
        sel = oracle_mod.select(w["A"]) if h == 1e-4 else sel
        errs, gst, ost = _check_parity(oracle_mod, w["A"], w["V"], w["t"], w["alpha"], s=sel["s"], xi=sel["xi"])
        print(f"h={h}: errs={errs} gpu={gst} oracle={ost}")


def test_advdiff2d_1024_full_size_fp64_and_fp32(oracle_mod):
    """The precision workload at full size (n = 1,048,576, Peclet 1e3, p = 4, r = 4, h = 1e-5), compared
    whole: FP64 at tol 2^-53 within 1e-12 and FP32 at tol 2^-24 within 5e-6 of the FP64 oracle."""
    oracle_mod.set_threads(0)
    w = wl.workload_advdiff2d_1024(1e-5, 2.0**-53)
    sel = oracle_mod.select(w["A"])
    ref, ost = oracle_mod.solve(w["A"], w["V"], w["t"], w["alpha"], TOL53, sel["s"], sel["xi"])
    W, gst = _gpu_solve(w["A"], w["V"], w["t"], w["alpha"], TOL53, sel["s"], sel["xi"])
    assert gst["status"] == 0 and gst["s_int"] == ost["s_int"] > 1
    assert max(_rel(W, ref)) <= 1e-12
    # FP32 with the GPU's Algorithm 1 for tol = 2^-24 (its s0 and f* let the FP32 solve cap each step's
    # norm); the exact result does not depend on (s, xi), so the FP64 oracle result above is the reference
    A32 = api.DeviceCSR.from_host(w["A"], dtype=torch.float32)
    P32 = api.select_params(A32, tol=TOL24)
    W32d, st32 = api.solve(A32, torch.as_tensor(w["V"]).float().cuda(), w["t"], w["alpha"], TOL24, P32)
    torch.cuda.synchronize()
    g32 = api.read_stats(st32)
    W32 = W32d.cpu().numpy()
    assert g32["status"] == 0
    assert max(_rel(W32, ref)) <= 5e-6
    print(f"advdiff 1024^2 h=1e-5: fp64 errs={_rel(W, ref)} fp32 errs={_rel(W32, ref)} s_int={gst['s_int']}")


@pytest.mark.parametrize("p,r", [(3, 2), (1, 4), (7, 2), (3, 4), (2, 3)])
def test_fp32_widths_against_fp64_oracle(oracle_mod, p, r):
    """FP32 tiles of 8, 16 and other widths (lane chunks of 8, 4, 2 or 1 floats) in the series and the
    recovery, with the GPU's Algorithm 1 at tol 2^-24, within 5e-6 of the FP64 oracle."""
    Acsr = wl.convection_diffusion(45, 2, 8.0)
    rng = np.random.default_rng(40 * p + r)
    V = rng.standard_normal((p + 1, Acsr.n))
    t = np.linspace(3e-3, 9e-3, r)
    alpha = np.linspace(0.6, 1.4, r)
    sel = oracle_mod.select(Acsr)
    ref, _ = oracle_mod.solve(Acsr, V, t, alpha, TOL53, sel["s"], sel["xi"])
    A32 = api.DeviceCSR.from_host(Acsr, dtype=torch.float32)
    P32 = api.select_params(A32, tol=TOL24)
    W, st = api.solve(A32, torch.as_tensor(V).float().cuda(), t, alpha, TOL24, P32)
    torch.cuda.synchronize()
    assert api.read_stats(st)["status"] == 0
    assert max(_rel(W.cpu().numpy(), ref)) <= 5e-6
