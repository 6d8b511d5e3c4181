"""expRK4s6 (eq. (1.4)) and the ADR operator on the CPU, without the library: the driver's stage inputs
(v_j, t_i, alpha_i for its four calls) combined with exact scalar phi values on a diagonal A give a
fourth-order method (step halving), and the ADR discretisation is second-order consistent."""
import math

import numpy as np
import scipy.sparse as sp

from paper_2509_26475_gb300 import exprk
from paper_2509_26475_gb300 import workloads as wl


def _phi(j, z):
    """phi_j(z) for real z: Taylor series near 0, else phi_j = (phi_{j-1} - 1/(j-1)!) / z upwards."""
    z = np.asarray(z, dtype=np.float64)
    out = np.empty_like(z)
    small = np.abs(z) < 0.5
    zs = z[small]
    acc = np.zeros_like(zs)
    for k in range(30):
        acc += zs**k / math.factorial(k + j)
    out[small] = acc
    zb = z[~small]
    f = np.exp(zb)
    for i in range(1, j + 1):
        f = (f - 1.0 / math.factorial(i - 1)) / zb
    out[~small] = f
    return out


def _combine(ci, lam):
    return [sum(a**j * _phi(j, t * lam) * ci.V[j] for j in range(len(ci.V))) for t, a in zip(ci.t, ci.alpha)]


def _step(u, h, lam, g):
    gu = g(u)
    hg = h * gu
    U2 = _combine(exprk.stage2_inputs(u, hg, h), lam)[0]
    D2 = g(U2) - gu
    U3, U4 = _combine(exprk.stage34_inputs(u, hg, D2, h), lam)
    D3, D4 = g(U3) - gu, g(U4) - gu
    U5, U6 = _combine(exprk.stage56_inputs(u, hg, D3, D4, h), lam)
    D5, D6 = g(U5) - gu, g(U6) - gu
    return _combine(exprk.final_inputs(u, hg, D5, D6, h), lam)[0]


def _integrate(u0, T, steps, lam, g):
    u = u0.copy()
    for _ in range(steps):
        u = _step(u, T / steps, lam, g)
    return u


def test_stage_inputs_give_fourth_order():
    lam = -np.linspace(1.0, 60.0, 7)
    g = exprk.adr_reaction(10.0)
    u0 = np.linspace(0.1, 0.9, 7)
    T = 0.5
    sols = [_integrate(u0, T, 8 * 2**k, lam, g) for k in range(5)]
    diffs = [np.abs(sols[k] - sols[k + 1]).max() for k in range(4)]
    orders = [math.log2(diffs[k] / diffs[k + 1]) for k in range(3)]
    assert all(3.7 <= o <= 4.4 for o in orders[1:]), orders


def test_scheme_is_exact_for_linear_problems():
    """With g = 0 every stage is phi_0(c h A) u_n, so one step is e^{hA} u_n exactly."""
    lam = -np.linspace(0.5, 30.0, 5)
    u0 = np.linspace(1.0, 2.0, 5)
    u1 = _step(u0, 0.3, lam, lambda u: 0.0 * u)
    assert np.allclose(u1, np.exp(0.3 * lam) * u0, rtol=1e-14, atol=0)


def test_adr_operator_is_second_order_consistent():
    errs = []
    for N in (40, 80, 160):
        A = wl.adr_operator(N)
        M = sp.csr_matrix((A.values, A.colidx, A.rowptr), shape=(A.n, A.n))
        x = np.arange(N) / N
        X, Y = np.meshgrid(x, x, indexing="xy")
        cx, cy = np.cos(np.pi * X / 2), np.cos(np.pi * Y / 2)
        sx, sy = np.sin(np.pi * X / 2), np.sin(np.pi * Y / 2)
        u = (cx * cy).ravel()  # u_x = 0 at x = 0, u = 0 at x = 1 (and likewise in y)
        exact = (wl.ADR_EPS * (-2 * (np.pi / 2) ** 2) * cx * cy
                 - wl.ADR_ALPHA * (-(np.pi / 2) * sx * cy - (np.pi / 2) * cx * sy)).ravel()
        errs.append(np.abs(M @ u - exact).max())
    assert 3.6 <= errs[0] / errs[1] <= 4.4 and 3.6 <= errs[1] / errs[2] <= 4.4, errs
    assert wl.adr_operator(100).n == 10_000
    u0 = wl.adr_initial(100)
    assert abs(u0.max() - 1.0) < 1e-3  # 256 x^2 y^2 (1-x)^2 (1-y)^2 peaks at 1 at (1/2, 1/2)
