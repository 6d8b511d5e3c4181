"""Algorithm 1 on the GPU against the oracle, through the C ABI.

The guard index r and s0 come from exact integer decisions and scaled norms: they must agree exactly
(r) and to rounding (s0).  The objective has a rounding-noise floor near its minimum (binomial
cancellation), so the minimisers can stop at different points: s must agree within 5 %, and the GPU's
xi* must be as good as the oracle's under the oracle's own objective (within 5 %).
"""
import math

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


def _gpu_select(Acsr, dtype=torch.float64, v=None, **kw):
    A = api.DeviceCSR.from_host(Acsr, dtype=dtype)
    vd = None if v is None else torch.as_tensor(v, dtype=torch.float64).cuda()
    P = api.select_params(A, v=vd, **kw)
    torch.cuda.synchronize()
    return api.read_params(P)


def _compare(oracle_mod, Acsr, v=None, dtype=torch.float64, tol=2.0**-53):
    g = _gpu_select(Acsr, dtype=dtype, v=v, tol=tol)
    Ao = Acsr if dtype == torch.float64 else wl.CSR(Acsr.n, Acsr.rowptr, Acsr.colidx,
                                                     Acsr.values.astype(np.float32).astype(np.float64))
    o = oracle_mod.select(Ao, v=v, tol=tol)
    assert g["status"] == 0, g
    assert g["r"] == o["r"], (g, o)
    assert abs(g["s0"] - o["s0"]) <= 1e-12 * o["s0"]
    assert abs(g["s"] - o["s"]) <= 0.05 * o["s"], (g, o)
    half = math.sqrt(Acsr.n) * o["s0"]
    assert -half <= g["xi"] <= half
    f_at_g, _, _ = oracle_mod.objective_at(Ao, [g["xi"]], v=v)
    assert f_at_g[0] <= 1.05 * o["f_star"], (f_at_g, g, o)
    return g, o


def test_laplacian_32(oracle_mod):
    g, o = _compare(oracle_mod, wl.laplacian_2d(32))
    assert g["r"] == 58


def test_convdiff3d_64_full_size(oracle_mod):
    oracle_mod.set_threads(0)
    g, o = _compare(oracle_mod, wl.workload_convdiff3d_64(1e-4)["A"])
    print("gpu", g, "oracle", o)


def test_given_vector_and_nonnormal(oracle_mod):
    rng = np.random.default_rng(1)
    n = 500
    Ad = np.triu(rng.standard_normal((n, n)), -2) + np.diag(np.linspace(-200.0, 1.0, n))
    v = rng.standard_normal(n)
    _compare(oracle_mod, wl.dense_to_csr(Ad), v=v)


def test_fp32_values_promoted(oracle_mod):
    _compare(oracle_mod, wl.convection_diffusion(50, 2, 30.0), dtype=torch.float32, tol=2.0**-24)


@pytest.mark.parametrize("d,r_exp", [([1e9, -3e8, 2.0, 0.5] * 100, 25), ([1e-9, 3e-10, -2e-9, 1e-12] * 100, 28)])
def test_guard_index(oracle_mod, d, r_exp):
    v = np.tile([0.3, -1.2, 0.7, 2.0], 100)
    g = _gpu_select(wl.diagonal(d), v=v)
    o = oracle_mod.select(wl.diagonal(d), v=v)
    assert g["r"] == o["r"] == r_exp
    assert abs(g["s0"] - o["s0"]) <= 1e-12 * o["s0"]


def test_zero_operator():
    Z = wl.CSR(300, np.zeros(301, dtype=np.int32), np.zeros(0, dtype=np.int32), np.zeros(0))
    g = _gpu_select(Z)
    assert g["status"] == 0 and g["r"] == 0 and g["xi"] == 0.0 and g["s"] == 1.0


def test_seeded_vector_matches_oracle_draw(oracle_mod):
    """Without v both sides draw components 2u-1 from splitmix64(seed, i): passing the oracle's draw
    explicitly must give the same guard index and s0."""
    A = wl.laplacian_2d(30)
    g1 = _gpu_select(A, seed=1234)
    g2 = _gpu_select(A, v=oracle_mod.unit_vector(A.n, 1234))
    assert g1["r"] == g2["r"] and g1["s0"] == g2["s0"] and g1["s"] == g2["s"]


def _ulp_diff(a: float, b: float) -> int:
    """Distance in units in the last place between two finite doubles of the same sign."""
    import struct

    ia = struct.unpack("<q", struct.pack("<d", a))[0]
    ib = struct.unpack("<q", struct.pack("<d", b))[0]
    return abs(ia - ib)


@pytest.mark.parametrize("m", [7, 40, 61, 128])
def test_objective_coefficients_against_exact_arithmetic(m):
    """The coefficients binom(m,k) z^(m-k) of Algorithm 1's objective as the selection kernel forms them
    (read back through phic_test_objective_coeffs), against exact rational arithmetic: binom(m, k) is the
    correctly rounded integer, z^(m-k) lies within one ulp of the exact power (double-double square and
    multiply), and the coefficient is their rounded product, so within 3 roundings of the exact one."""
    import ctypes
    from fractions import Fraction

    lib = capi.load()
    rng = np.random.default_rng(m)
    zs = [0.0, 1.0, -1.0, 0.5, -2.75] + list(rng.uniform(-1.0, 1.0, 12) * 10.0 ** rng.uniform(-2.0, 1.5, 12))
    out = torch.empty(3 * (m + 1), dtype=torch.float64, device="cuda")
    exact_pow = 0
    total = 0
    for z in zs:
        capi.check(lib.phic_test_objective_coeffs(m, ctypes.c_double(float(z)), out.data_ptr(), None),
                   "phic_test_objective_coeffs")
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        coef, pw, bn = o[: m + 1], o[m + 1: 2 * (m + 1)], o[2 * (m + 1):]
        for k in range(m + 1):
            b_exact = math.comb(m, k)
            assert bn[k] == float(b_exact), (m, k)
            p_exact = Fraction(float(z)) ** (m - k)
            try:
                p_ref = float(p_exact)
            except OverflowError:
                continue
            if p_ref == 0.0 or abs(p_ref) < 1e-290:
                assert abs(pw[k]) <= 1e-290
                continue
            assert _ulp_diff(float(pw[k]), p_ref) <= 1, (m, z, k, pw[k], p_ref)
            exact_pow += int(float(pw[k]) == p_ref)
            total += 1
            assert float(coef[k]) == float(bn[k]) * float(pw[k])  # one rounding of the two doubles' product
            c_exact = b_exact * p_exact
            assert abs(Fraction(float(coef[k])) - c_exact) <= abs(c_exact) * Fraction(3, 2**53), (m, z, k)
    print(f"m={m}: {exact_pow} of {total} powers correctly rounded, the rest within one ulp")
