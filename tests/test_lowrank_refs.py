"""The long-double closed form used by the GPU low-rank tests (where mpmath is not installed) against the
mpmath form, and against the oracle on the dense matrix U M U^T (paper's third experiment, Section 6)."""
import numpy as np
import pytest

import refs
from paper_2509_26475_gb300 import workloads as wl

M3 = np.array([[0.0, 1e-8, 0.0], [-(2e10 + 4e8 / 6), -3.0, 2e10], [200.0 / 3, 0.0, -200.0 / 3]])
CORES = {"M1": np.array([[0.0, 10.0], [-10.0, 0.0]]), "M2": np.array([[-1.0, 1e5], [0.0, -10.0]]), "M3": M3}


@pytest.mark.parametrize("core,t", [("M1", 0.1), ("M1", 10.0), ("M2", 0.1), ("M2", 1.0), ("M3", 1e-5), ("M3", 1e-3)])
def test_long_double_phi_matrices_match_mpmath(core, t):
    pytest.importorskip("mpmath")
    X = t * CORES[core]
    a = refs.phi_matrices_ld(X, 5)
    b = refs.phi_matrices(X, 5, dps=60)
    # M3's scaling and squaring (||X|| up to 4e7) costs ~1e-11 in x86 80-bit long double (IEEE quad on
    # aarch64 is far tighter); the paper's smallest M3 error is 2.4e-10
    bar = 1e-10 if core == "M3" else 1e-12
    for j in range(6):
        A = np.asarray(a[j], dtype=np.float64)
        assert np.abs(A - b[j]).max() <= bar * np.abs(b[j]).max(), (core, t, j)


def test_long_double_closed_form_matches_the_oracle(oracle_mod):
    n, p = 160, 3
    M = CORES["M1"]
    Ad, U = wl.low_rank_dct(n, M)
    W = U @ M.T
    V = np.random.default_rng(4).standard_normal((p + 1, n))
    A = wl.dense_to_csr(Ad, keep_zeros=True)
    sel = oracle_mod.select(A)
    for t, alpha in ((0.7, 1.0), (0.3, 1.7)):
        out, _ = oracle_mod.solve(A, V, [t], [alpha], 2.0**-53, sel["s"], sel["xi"])
        ref = refs.low_rank_comb_ld(U, W, M, V, t, alpha)
        assert refs.rel2(out[0], ref) < 1e-12
