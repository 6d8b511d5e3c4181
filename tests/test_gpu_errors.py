"""Error paths of the C ABI on the device.  None of these faults or hangs a GPU: bad indices are
checked before use, and the timeout case makes a bounded barrier wait expire (block 0 leaves before
arriving), after which every block returns and the context stays usable."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2509_26475_gb300 import api, capi
from paper_2509_26475_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2509_26475_gb300 import build

    build.build()
    capi.load()


def _solve_status(Acsr, V, t=(1e-3,), alpha=(1.0,), s=100.0, xi=-10.0, **kw):
    A = api.DeviceCSR.from_host(Acsr)
    Vd = torch.as_tensor(V).cuda()
    P = api.set_params(xi, s)
    W, st = api.solve(A, Vd, list(t), list(alpha), 2.0**-53, P, **kw)
    torch.cuda.synchronize()
    return api.read_stats(st)


def test_bad_column_index():
    A = wl.laplacian_2d(30)
    bad = wl.CSR(A.n, A.rowptr, A.colidx.copy(), A.values)
    bad.colidx[777] = A.n + 5
    st = _solve_status(bad, np.ones((2, A.n)))
    assert st["status"] == capi.PHIC_INVALID_ARG
    A2 = api.DeviceCSR.from_host(bad)
    P = api.select_params(A2)
    torch.cuda.synchronize()
    assert api.read_params(P)["status"] == capi.PHIC_INVALID_ARG


def test_bad_rowptr():
    A = wl.laplacian_2d(30)
    rp = A.rowptr.copy()
    rp[100], rp[101] = rp[101], rp[100]
    st = _solve_status(wl.CSR(A.n, rp, A.colidx, A.values), np.ones((2, A.n)))
    assert st["status"] == capi.PHIC_INVALID_ARG


def test_term_cap_and_nonfinite():
    A = wl.laplacian_2d(30)
    st = _solve_status(A, np.ones((2, A.n)), t=(0.1,), max_terms=3)
    assert st["status"] == capi.PHIC_TERM_CAP
    V = np.ones((2, A.n))
    V[1, 17] = np.nan
    st = _solve_status(A, V)
    assert st["status"] == capi.PHIC_NONFINITE


def test_timeout_is_reported_and_context_survives():
    lib = capi.load()
    A = wl.laplacian_2d(64)  # 4096 rows: several blocks
    lib.phic_set_spin_limit_ms(200.0)
    try:
        lib.phic_set_test_fault(1)
        st = _solve_status(A, np.ones((2, A.n)))
        assert st["status"] == capi.PHIC_TIMEOUT
    finally:
        lib.phic_set_test_fault(0)
        lib.phic_set_spin_limit_ms(2000.0)
    st = _solve_status(A, np.ones((2, A.n)))
    assert st["status"] == capi.PHIC_OK


def test_host_argument_checks():
    lib = capi.load()
    A = api.DeviceCSR.from_host(wl.laplacian_2d(10))
    V = torch.ones((3, A.n), dtype=torch.float64, device="cuda")
    P = api.set_params(0.0, 1.0)
    with pytest.raises(ValueError):  # the binding rejects FP64 V against FP32 values
        api.solve(A.astype(torch.float32), V, [1.0], [1.0], 1e-10, P)
    c32 = A.astype(torch.float32).struct()
    t1 = (ctypes.c_double * 1)(1.0)
    W = torch.empty((1, A.n), dtype=torch.float64, device="cuda")
    ws = torch.empty(api.solve_workspace_bytes(A.n, A.nnz, 2, 1, 0), dtype=torch.uint8, device="cuda")
    assert lib.phic_solve(ctypes.byref(c32), 2, 1, V.data_ptr(), t1, t1, 1e-10, P.data_ptr(), 0, 0, W.data_ptr(),
                          ws.data_ptr(), ws.numel(), None, 0, None) == capi.PHIC_INVALID_ARG  # prec mismatch
    with pytest.raises(capi.PhicError):  # r above the limit
        api.solve(A, V, np.ones(17), np.ones(17), 1e-10, P)
    small = torch.empty(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(capi.PhicError) as ei:
        api.solve(A, V, [1.0], [1.0], 1e-10, P, workspace=small)
    assert ei.value.status == capi.PHIC_WORKSPACE_TOO_SMALL
    c = A.struct()
    t = (ctypes.c_double * 1)(1.0)
    assert lib.phic_solve(ctypes.byref(c), 2, 1, V.data_ptr(), t, t, -1.0, P.data_ptr(), 0, 0, V.data_ptr(),
                          small.data_ptr(), small.numel(), None, 0, None) == capi.PHIC_INVALID_ARG
