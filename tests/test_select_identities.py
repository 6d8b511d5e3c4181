"""Two numerical facts Algorithm 1's kernel relies on, checked on the host.

1. The guard's bound max_j log binom(m, j) sits at the middle index (both middle indices for odd m):
   neighbouring j differ by at least log(1 + 2/m), far above the rounding of lgamma, so evaluating the
   middle indices in the same form gives the full scan's value.
2. z^e by square and multiply carried in double-double (Dekker's exact product through an FMA) and
   rounded once is correctly rounded for the objective's coefficients binom(m, k) z^(m-k); the method
   is mirrored here with an exact FMA (rational arithmetic)."""
import math
import random
from fractions import Fraction


def test_largest_log_binomial_at_the_middle():
    for m in range(1, 129):
        terms = [math.lgamma(m + 1.0) - math.lgamma(j + 1.0) - math.lgamma(m - j + 1.0) for j in range(m + 1)]
        mid = [terms[j] for j in range(m // 2, (m + 1) // 2 + 1)]
        assert max(terms) == max(mid), m
        off = [terms[j] for j in range(m + 1) if not m // 2 <= j <= (m + 1) // 2]
        if off:  # every other term lies at least log(1 + 2/m) below, far above lgamma's rounding
            assert max(terms) - max(off) >= math.log1p(2.0 / m) * (1.0 - 1e-9), m


def _fma(a, b, c):
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def _dd_mul(ah, al, bh, bl):
    p = ah * bh
    if not math.isfinite(p):
        return p, 0.0
    e = _fma(ah, bh, -p) + (ah * bl + al * bh)
    s = p + e
    return s, e - (s - p)


def _pow_int(z, e):
    rh, rl, bh, bl = 1.0, 0.0, z, 0.0
    while e > 0:
        if e & 1:
            rh, rl = _dd_mul(rh, rl, bh, bl)
        e >>= 1
        if e:
            bh, bl = _dd_mul(bh, bl, bh, bl)
    return rh + rl if math.isfinite(rh) else rh


def test_double_double_integer_power_is_correctly_rounded():
    rng = random.Random(7)
    for _ in range(120):
        z = rng.uniform(-3.0, 3.0) * 10.0 ** rng.uniform(-2.0, 1.0)
        for e in range(0, 129, 3):
            exact = Fraction(z) ** e
            try:
                ref = float(exact)
            except OverflowError:
                continue
            if ref == 0.0 or not math.isfinite(ref) or abs(ref) < 1e-300:
                continue
            assert _pow_int(z, e) == ref, (z, e)
    assert _pow_int(1e200, 3) == math.inf and _pow_int(-1e200, 3) == -math.inf
