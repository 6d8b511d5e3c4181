"""Every copy format of B the setup can pick (DIA with 5, 7 or another number of diagonals, ELL, CSR
order), each with its own loop nest in the single-instance kernels, against the oracle in FP64 (bar
1e-12 at tol 2^-53) and in FP32 (bar 5e-6 at tol 2^-24, against the FP64 oracle), for block widths
that take every lane chunk (1, 2, 4 and 8 columns, and 3 and 5: widths 12 and 20).  phic_stats reports the format the solve used.
Both precisions run with the oracle's (s, xi), so that s_int >= 2 and the recovery loop runs."""
import numpy as np
import pytest
import torch

from paper_2509_26475_gb300 import api
from paper_2509_26475_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL53, TOL24 = 2.0**-53, 2.0**-24


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2509_26475_gb300 import build, capi

    build.build()
    capi.load()
    torch.cuda.set_device(0)


def _rel(W, ref):
    W = np.asarray(W, dtype=np.float64)
    return [float(np.linalg.norm(W[i] - ref[i]) / np.linalg.norm(ref[i])) for i in range(ref.shape[0])]


# (name, builder, expected format, expected slots, t scale)
CASES = [
    ("dia5", lambda: wl.convection_diffusion(37, 2, 6.0), "dia", 5, 4e-3),
    ("dia7", lambda: wl.convection_diffusion(13, 3, 6.0), "dia", 7, 2e-2),
    ("dia3", lambda: wl.convection_diffusion(1500, 1, 6.0), "dia", 3, 1e-5),
    ("ell", lambda: wl.graph_operator(2500, 6, 11), "ell", 7, 2.0),
    ("csr", lambda: wl.graph_operator(2600, 6, 12, hubs=20, hub_degree=80), "csr", 0, 0.3),
]
WIDTHS = [(3, 2), (4, 4), (2, 4), (0, 3), (1, 1)]


@pytest.mark.parametrize("name,make,fmt,slots,tscale", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("p,r", WIDTHS)
def test_format_fp64(oracle_mod, name, make, fmt, slots, tscale, p, r):
    Acsr = make()
    rng = np.random.default_rng(7 * p + r)
    V = rng.standard_normal((p + 1, Acsr.n))
    t = tscale * np.linspace(1.0, 0.5, r)  # t_1 = tscale for every r
    alpha = np.linspace(0.7, 1.3, r)
    sel = oracle_mod.select(Acsr)
    ref, ost = oracle_mod.solve(Acsr, V, t, alpha, TOL53, sel["s"], sel["xi"])
    A = api.DeviceCSR.from_host(Acsr, dtype=torch.float64)
    P = api.set_params(sel["xi"], sel["s"])
    W, st = api.solve(A, torch.as_tensor(V).cuda(), t, alpha, TOL53, P)
    torch.cuda.synchronize()
    gst = api.read_stats(st)
    assert gst["status"] == 0, gst
    assert (gst["op_format"], gst["op_slots"]) == (fmt, slots), gst
    assert gst["s_int"] == ost["s_int"] and gst["s_int"] >= 2, (gst, ost)
    assert max(_rel(W.cpu().numpy(), ref)) <= 1e-12


@pytest.mark.parametrize("name,make,fmt,slots,tscale", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("p,r", WIDTHS)
def test_format_fp32(oracle_mod, name, make, fmt, slots, tscale, p, r):
    Acsr = make()
    rng = np.random.default_rng(7 * p + r)
    V = rng.standard_normal((p + 1, Acsr.n))
    t = tscale * np.linspace(1.0, 0.5, r)  # t_1 = tscale for every r
    alpha = np.linspace(0.7, 1.3, r)
    sel = oracle_mod.select(Acsr)
    ref, _ = oracle_mod.solve(Acsr, V, t, alpha, TOL53, sel["s"], sel["xi"])
    A = api.DeviceCSR.from_host(Acsr, dtype=torch.float32)
    P = api.set_params(sel["xi"], sel["s"])  # the FP64 scaling: the same outer steps as the FP64 test
    W, st = api.solve(A, torch.as_tensor(V).float().cuda(), t, alpha, TOL24, P)
    torch.cuda.synchronize()
    gst = api.read_stats(st)
    assert gst["status"] == 0, gst
    assert (gst["op_format"], gst["op_slots"]) == (fmt, slots), gst
    assert gst["s_int"] >= 2, gst
    assert max(_rel(W.cpu().numpy(), ref)) <= 5e-6
