"""A numerical fact Algorithm 1's kernel relies on, checked on the host: the guard's bound
max_j log binom(m, j) sits at the middle index (both middle indices for odd m).  Neighbouring j differ by
at least log(1 + 2/m), far above the rounding of lgamma, so evaluating the middle indices in the same form
gives the full scan's value.  (The objective's coefficients binom(m, k) z^(m-k) are checked as the device
forms them, against exact arithmetic, in test_gpu_select.py.)"""
import math


def test_largest_log_binomial_at_the_middle():
    for m in range(1, 129):
        terms = [math.lgamma(m + 1.0) - math.lgamma(j + 1.0) - math.lgamma(m - j + 1.0) for j in range(m + 1)]
        mid = [terms[j] for j in range(m // 2, (m + 1) // 2 + 1)]
        assert max(terms) == max(mid), m
        off = [terms[j] for j in range(m + 1) if not m // 2 <= j <= (m + 1) // 2]
        if off:  # every other term lies at least log(1 + 2/m) below, far above lgamma's rounding
            assert max(terms) - max(off) >= math.log1p(2.0 / m) * (1.0 - 1e-9), m
