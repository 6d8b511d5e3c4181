"""phic_solve_noalloc against phic_solve, through the C ABI.

phic_solve_noalloc serves callers that cannot allocate device memory (a plug-in inside a host
application that owns every allocation, a latency-critical loop that cannot pay for cudaMalloc's
synchronisation, a system that allocates only at start-up): it takes no workspace and keeps its scratch
in a static device array shared by all calls.  Its output must match phic_solve's within the FP64 parity
tolerance of the other tests (1e-12 relative) on consecutive calls, whatever the previous call left in
the shared array.  This file sorts last so that a run stopping at the first failure has already run
every other test; it also passes alone in a fresh process (the first call looks up the array).
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2509_26475_gb300 import api, capi
from paper_2509_26475_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL53 = 2.0**-53


def _noalloc(lib, A, V, p, t, alpha, P, flags=0):
    r = len(t)
    W = torch.empty((r, A.n), dtype=V.dtype, device=V.device)
    st = api.new_stats(V.device)
    c = A.struct()
    ta = (ctypes.c_double * r)(*t)
    aa = (ctypes.c_double * r)(*alpha)
    rc = lib.phic_solve_noalloc(ctypes.byref(c), p, r, V.data_ptr(), ta, aa, TOL53, P.data_ptr(), flags, 0,
                                W.data_ptr(), st.data_ptr(), A.prec, torch.cuda.current_stream().cuda_stream)
    return rc, W, st


def test_noalloc_matches_solve_on_consecutive_calls():
    from paper_2509_26475_gb300 import build

    build.build()
    lib = capi.load()
    torch.cuda.set_device(0)
    rng = np.random.default_rng(77)
    cases = [
        (wl.convection_diffusion(60, 2, 10.0), 3, [2e-3, 1e-3], [0.5, 1.0 / 3.0]),
        (wl.convection_diffusion(60, 2, 10.0), 3, [2e-3, 1e-3], [0.5, 1.0 / 3.0]),
        (wl.laplacian_2d(45), 2, [4e-3], [1.0]),
    ]
    for Acsr, p, t, alpha in cases:
        A = api.DeviceCSR.from_host(Acsr)
        V = torch.as_tensor(rng.standard_normal((p + 1, Acsr.n))).cuda()
        P = api.select_params(A)
        W_ref, st_ref = api.solve(A, V, t, alpha, TOL53, P)
        rc, W, st = _noalloc(lib, A, V, p, t, alpha, P)
        assert rc == capi.PHIC_OK
        torch.cuda.synchronize()
        assert api.read_stats(st_ref)["status"] == 0 and api.read_stats(st)["status"] == 0
        a, b = W.cpu().numpy(), W_ref.cpu().numpy()
        for i in range(len(t)):
            assert np.linalg.norm(a[i] - b[i]) / np.linalg.norm(b[i]) <= 1e-12
        assert api.read_stats(st)["recovery_terms"] == api.read_stats(st_ref)["recovery_terms"]


def test_noalloc_rejects_problems_above_the_static_size():
    lib = capi.load()
    Acsr = wl.laplacian_3d(48)  # 110,592 rows: FP64 p = 3, r = 2 needs about 61 MB of scratch
    assert api.solve_workspace_bytes(Acsr.n, Acsr.nnz, 3, 2, capi.PHIC_F64) > capi.PHIC_NOALLOC_MAX_BYTES
    A = api.DeviceCSR.from_host(Acsr)
    V = torch.zeros((4, Acsr.n), dtype=torch.float64, device="cuda")
    P = api.set_params(0.0, 1.0)
    rc, W, st = _noalloc(lib, A, V, 3, [1e-3, 2e-3], [1.0, 1.0], P)
    assert rc == capi.PHIC_WORKSPACE_TOO_SMALL
