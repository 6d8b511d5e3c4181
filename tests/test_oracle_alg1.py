"""Pins of the oracle's Algorithm 1 (scaling s and shift xi*, Section 3).

The objective f(xi) is evaluated by the binomial sum the paper prints; near its minimum that sum
cancels heavily, so its computed value has a rounding floor and the location of xi* is not fixed
to more than a few digits ("parity unpinned" for xi* itself).  What is pinned:
  * the guard index r and the log-norms L_k = log ||A^k v|| against closed forms on diagonal A;
  * s0 = geometric mean of the last growth factors, from the closed-form L_k;
  * f(xi) s0 = ||(A - xi I)^m v||^(1/m) where the binomial sum has no cancellation (A >= 0, xi < 0);
  * the Brent minimiser on functions with known minimisers;
  * s = s0 f(xi*) / (tol m!)^(1/m) and the power-of-two equivariance A -> 2A (xi, s double);
  * on the 2-D Laplacian, xi* lies inside the spectrum and s (tol m!)^(1/m) is within [0.9, 3] times the
    spectral half-width (the noise floor only inflates f).
"""
import math

import numpy as np
import pytest

from paper_2509_26475_gb300 import workloads as wl

DBL_MAX_LOG = math.log(np.finfo(np.float64).max)
DBL_MIN_LOG = math.log(np.finfo(np.float64).tiny)


def _closed_form_logs(d, v, m):
    import mpmath as mp

    with mp.workdps(50):
        v = [mp.mpf(x) for x in v]
        nv = mp.sqrt(sum(x * x for x in v))
        v = [x / nv for x in v]
        return [float(mp.log(mp.sqrt(sum((mp.mpf(di) ** k * vi) ** 2 for di, vi in zip(d, v))))) for k in range(m + 1)]


def _expected_r(L, m, delta=0.8):
    gmax, gmin = delta * DBL_MAX_LOG, delta * DBL_MIN_LOG
    lmax = max(math.lgamma(m + 1) - math.lgamma(j + 1) - math.lgamma(m - j + 1) for j in range(m + 1))
    r = 0
    for k in range(1, m + 1):
        if L[k] + 0.5 * math.log(k + 1) + lmax > gmax or L[k] < gmin:
            break
        r = k
    return r


@pytest.mark.parametrize("d", [[1e9, -3e8, 2.0, 0.5], [1e-9, 3e-10, -2e-9, 1e-12], [3.0, -2.0, 0.1, 1.5]])
def test_guard_index_and_lognorms(oracle_mod, d):
    v = np.array([0.3, -1.2, 0.7, 2.0])
    m = 61
    L = _closed_form_logs(d, v, m)
    r_exp = _expected_r(L, m)
    res = oracle_mod.select(wl.diagonal(d), m=m, v=v)
    assert res["r"] == r_exp
    np.testing.assert_allclose(res["L"], L[: r_exp + 1], rtol=1e-12, atol=1e-12)
    jr = max(2, r_exp - 5)
    if r_exp - jr <= 0:
        jr = max(0, r_exp - 1)
    s0 = math.exp((L[r_exp] - L[jr]) / (r_exp - jr))
    assert abs(res["s0"] - s0) <= 1e-12 * s0
    if d[0] == 1e9:
        assert r_exp == 25  # 20.72 k - 2.1 + log(k+1)/2 + 39.9 > 567.8 first at k = 26
    if d[0] == 1e-9:
        assert r_exp == 28  # dominated by |-2e-9|: -20.03 k - 1.26 < -566.7 first at k = 29


def test_objective_without_cancellation(oracle_mod):
    """A >= 0 and xi < 0: every binomial term has the same sign, so f is accurate; compare with
    ||(A - xi I)^m v||^(1/m) / s0 in mpmath."""
    import mpmath as mp

    d = np.array([0.5, 2.0, 3.5, 7.0, 1.25])
    v = np.array([1.0, -0.4, 0.25, 0.8, -1.1])
    m = 61
    xis = np.array([-0.5, -3.0, -20.0])
    f, s0, r = oracle_mod.objective_at(wl.diagonal(d), xis, m=m, v=v)
    assert r == m
    with mp.workdps(60):
        nv = mp.sqrt(sum(mp.mpf(x) ** 2 for x in v))
        for xi, fx in zip(xis, f):
            nu = mp.sqrt(sum(((mp.mpf(di) - mp.mpf(xi)) ** m * mp.mpf(vi) / nv) ** 2 for di, vi in zip(d, v)))
            expect = float(nu ** (mp.mpf(1) / m)) / s0
            assert abs(fx - expect) <= 1e-13 * expect


@pytest.mark.parametrize("top", [1e9, 3.7e7])
def test_objective_through_the_extended_basis(oracle_mod, top):
    """The extension V_k = A V_(k-1) / s0 for k = r+1..m (Algorithm 1 after the guard): a diagonal A >= 0
    whose top eigenvalue is large enough that the guard stops the power chain well before m = 61, and
    xi < 0, so every binomial term of f has one sign and f is accurate.  f(xi) must equal
    ||(A - xi I)^m v||^(1/m) / s0 (mpmath, 60 digits), which holds only when every extended column carries
    exactly one more factor A / s0: a dropped or repeated 1/s0 moves f by a factor s0^(j/m) for some
    j >= 1, at least about 1.3 here."""
    import mpmath as mp

    d = np.array([top, 0.5, 2.0, 3.5e3, 7.0, 0.0, 41.0])
    v = np.array([0.7, -1.0, 0.25, 0.8, -1.1, 0.3, 0.05])
    m = 61
    xis = np.array([-1.0e3, -1.0e8, -2.5 * top])
    f, s0, r = oracle_mod.objective_at(wl.diagonal(d), xis, m=m, v=v)
    assert 2 <= r < m - 20, r  # most of the basis comes from the extension
    assert s0 > 0.5 * top  # the growth factor of the dominant eigenvalue
    with mp.workdps(60):
        nv = mp.sqrt(sum(mp.mpf(x) ** 2 for x in v))
        for xi, fx in zip(xis, f):
            nu = mp.sqrt(sum(((mp.mpf(di) - mp.mpf(xi)) ** m * mp.mpf(vi) / nv) ** 2 for di, vi in zip(d, v)))
            expect = float(nu ** (mp.mpf(1) / m)) / s0
            assert abs(fx - expect) <= 1e-13 * expect, (xi, fx, expect)


def test_objective_at_zero_shift_is_scaled_power_norm(oracle_mod):
    """f(0) = ||A^m v||^(1/m) / s0 (only the k = m term survives; no cancellation) for any A."""
    import mpmath as mp

    d = np.array([-4.0, 1.0, 2.5, -0.3])
    v = np.array([0.2, 0.9, -0.5, 1.3])
    m = 40
    f, s0, r = oracle_mod.objective_at(wl.diagonal(d), [0.0], m=m, v=v)
    with mp.workdps(50):
        nv = mp.sqrt(sum(mp.mpf(x) ** 2 for x in v))
        nu = mp.sqrt(sum((mp.mpf(di) ** m * mp.mpf(vi) / nv) ** 2 for di, vi in zip(d, v)))
        expect = float(nu ** (mp.mpf(1) / m)) / s0
    assert abs(f[0] - expect) <= 1e-13 * expect


@pytest.mark.parametrize("fn,a,b,xstar", [
    (lambda x: (x - 1.234) ** 2 + 3.0, -10.0, 10.0, 1.234),
    (lambda x: math.cos(x), 2.0, 5.0, math.pi),
    (lambda x: abs(x + 0.3) ** 0.5, -2.0, 7.0, -0.3),
    (lambda x: math.exp(x) - 3.0 * x, -4.0, 6.0, math.log(3.0)),
    (lambda x: x, 1.0, 2.0, 1.0),  # monotone: converges to the left end
])
def test_brent_finds_known_minimisers(oracle_mod, fn, a, b, xstar):
    x, fx, ne = oracle_mod.minimize(fn, a, b, tabs=1e-9, max_evals=200)
    assert abs(x - xstar) <= 1e-6 * max(1.0, abs(xstar)), (x, xstar)
    assert ne < 200


def test_scaling_formula_and_power_of_two_equivariance(oracle_mod):
    rng = np.random.default_rng(4)
    n = 30
    Ad = np.diag(np.linspace(-3.0, -0.1, n)) + 0.2 * np.triu(rng.standard_normal((n, n)), 1)
    A = wl.dense_to_csr(Ad)
    m, tol = 61, 2.0**-53
    r1 = oracle_mod.select(A, m=m, tol=tol)
    assert r1["r"] == m
    lg = (math.log(tol) + math.lgamma(m + 1)) / m
    assert abs(r1["s"] - r1["s0"] * r1["f_star"] / math.exp(lg)) <= 1e-14 * r1["s"]
    r2 = oracle_mod.select(A.scaled(2.0), m=m, tol=tol)
    assert abs(r2["s0"] - 2.0 * r1["s0"]) <= 1e-12 * r2["s0"]
    # the objective's rounding floor lets the minimiser take a slightly different path: 5 % band
    assert abs(r2["s"] - 2.0 * r1["s"]) <= 0.05 * r2["s"]
    assert abs(r2["xi"] - 2.0 * r1["xi"]) <= 0.05 * math.sqrt(n) * r2["s0"]


def test_laplacian_shift_and_scale_bounds(oracle_mod):
    N = 32
    A = wl.laplacian_2d(N)
    h = 1.0 / (N + 1)
    lam1 = -(4.0 / h**2) * np.sin(np.arange(1, N + 1) * np.pi * h / 2.0) ** 2
    lmin, lmax = 2 * lam1.min(), 2 * lam1.max()
    half = 0.5 * (lmax - lmin)
    res = oracle_mod.select(A)
    assert lmin <= res["xi"] <= lmax
    m, tol = 61, 2.0**-53
    scaled = res["s"] * math.exp((math.log(tol) + math.lgamma(m + 1)) / m)
    assert 0.9 * half <= scaled <= 3.0 * half, (scaled, half)
    assert res["r"] == 58  # guard index of the 32 x 32 Laplacian (both norms scaled)


def test_zero_power_gives_unit_parameters(oracle_mod):
    """A v = 0 (reading: nothing accepted): xi = 0, s = 1."""
    Z = wl.CSR(5, np.arange(6, dtype=np.int32), np.arange(5, dtype=np.int32), np.zeros(5))
    res = oracle_mod.select(Z)
    assert res["r"] == 0 and res["xi"] == 0.0 and res["s"] == 1.0


def test_unit_vector_is_splitmix64(oracle_mod):
    """Known answers of the published splitmix64 sequence from state 0: 0xe220a8397b1dcdaf,
    0x6e789e6aa1b965f4; component = 2 * (z >> 11) * 2^-53 - 1."""
    v = oracle_mod.unit_vector(2, 0)
    for z, x in zip([0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4], v):
        assert x == 2.0 * ((z >> 11) * 2.0**-53) - 1.0
