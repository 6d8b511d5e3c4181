"""Independent references that pin the oracle (and, through it, the CUDA path).

None of these follow the paper's algorithms: each computes the same mathematical object by a
different route, so that a slip in the oracle (a dropped term, a wrong sign or index, a transposed
operand) shows up as a mismatch.

  * ``aug_comb``          -- w = [I 0] exp([[tA, W],[0, J_p(0)]]) [v0; e_p] with W = [a^p v_p .. a v_1]
                             (the augmented-matrix formula of the paper's first experiment, Section 5,
                             with tA and the weights a^j folded in), by SciPy's expm or by a
                             scaling-and-squaring Taylor exponential in numpy long double.
  * ``phi_scalar``        -- phi_j(z) in mpmath (series for |z| < 1, the recurrence
                             phi_{j+1}(z) = (phi_j(z) - 1/j!)/z otherwise).
  * ``laplacian_2d_comb`` -- closed form for the 5-point Dirichlet Laplacian through its sine-transform
                             eigenbasis.
  * ``low_rank_comb``     -- closed form for A = U M U^T (the paper's third experiment, Section 5) with
                             phi_{j+1}(tM) from an mpmath exponential of a small block matrix.
"""
from __future__ import annotations

import math

import numpy as np


def rel2(x, ref):
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.linalg.norm(x - ref) / np.linalg.norm(ref))


def _aug_matrix(Ad, V, t, a, dtype):
    n = Ad.shape[0]
    p = V.shape[0] - 1
    M = np.zeros((n + p, n + p), dtype=dtype)
    M[:n, :n] = np.asarray(Ad, dtype=dtype) * dtype(t)
    for c in range(p):  # column c holds a^{p-c} v_{p-c}
        j = p - c
        M[:n, n + c] = np.asarray(V[j], dtype=dtype) * (dtype(a) ** j)
    for c in range(p - 1):
        M[n + c, n + c + 1] = 1
    x = np.zeros(n + p, dtype=dtype)
    x[:n] = np.asarray(V[0], dtype=dtype)
    if p > 0:
        x[n + p - 1] = 1
    return M, x


def expm_longdouble(M):
    """exp(M) by scaling and squaring of a degree-30 Taylor polynomial in numpy long double."""
    M = np.asarray(M, dtype=np.longdouble)
    nrm = float(np.max(np.sum(np.abs(M), axis=0))) if M.size else 0.0
    k = 0
    if nrm > 0.125:
        k = int(math.ceil(math.log2(nrm / 0.125)))
    X = M / np.longdouble(2.0) ** k
    I = np.eye(M.shape[0], dtype=np.longdouble)
    E = I.copy()
    term = I.copy()
    for q in range(1, 31):
        term = (term @ X) / np.longdouble(q)
        E = E + term
    for _ in range(k):
        E = E @ E
    return E


def aug_comb(Ad, V, t, a, method="scipy"):
    """sum_j a^j phi_j(tA) v_j for dense A via the augmented exponential."""
    Ad = np.asarray(Ad)
    V = np.asarray(V)
    n = Ad.shape[0]
    if method == "scipy":
        import scipy.linalg as sl

        M, x = _aug_matrix(Ad, V, t, a, np.float64)
        return (sl.expm(M) @ x)[:n]
    M, x = _aug_matrix(Ad, V, t, a, np.longdouble)
    return (expm_longdouble(M) @ x)[:n].astype(np.float64)


def phi_scalar(j: int, z, dps: int = 60):
    """phi_j(z) as an mpmath number (z real or complex)."""
    import mpmath as mp

    with mp.workdps(dps):
        z = mp.mpmathify(z)
        if abs(z) < 1:
            s = mp.mpf(0)
            term = 1 / mp.factorial(j)
            k = 0
            while True:
                s += term
                k += 1
                term = term * z / (k + j)
                if abs(term) < mp.mpf(10) ** (-dps):
                    break
            return s
        ph = mp.exp(z)
        for q in range(j):
            ph = (ph - 1 / mp.factorial(q)) / z
        return ph


def diag_comb(d, V, t, a):
    """Closed form for diagonal A = diag(d): w[k] = sum_j a^j phi_j(t d_k) v_j[k]."""
    d = np.asarray(d, dtype=np.float64)
    p = V.shape[0] - 1
    w = np.zeros(d.size)
    for k in range(d.size):
        acc = 0.0
        for j in range(p + 1):
            acc += float(a) ** j * float(phi_scalar(j, float(t) * d[k])) * V[j, k]
        w[k] = acc
    return w


def dst_basis(N: int) -> np.ndarray:
    """Orthonormal eigenvectors of the 1-D Dirichlet second difference (sine transform)."""
    i = np.arange(1, N + 1)[:, None]
    k = np.arange(1, N + 1)[None, :]
    return np.sqrt(2.0 / (N + 1)) * np.sin(np.pi * i * k / (N + 1))


def laplacian_2d_comb(N: int, V, t, a):
    """Closed form for the 5-point Dirichlet Laplacian on an N x N grid, h = 1/(N+1)."""
    h = 1.0 / (N + 1)
    lam1 = -(4.0 / h**2) * np.sin(np.arange(1, N + 1) * np.pi * h / 2.0) ** 2
    Q = dst_basis(N)
    lam = lam1[:, None] + lam1[None, :]  # lam[kx, ky]
    p = V.shape[0] - 1
    phis = np.zeros((p + 1, N, N))
    import mpmath as mp

    for j in range(p + 1):
        f = np.vectorize(lambda z: float(phi_scalar(j, z, dps=40)))
        phis[j] = f(float(t) * lam)
    w = np.zeros((N, N))
    for j in range(p + 1):
        X = V[j].reshape(N, N)  # X[y, x]; x fastest in the row ordering
        C = Q.T @ X @ Q         # coefficients C[ky, kx]
        w += float(a) ** j * (Q @ (phis[j].T * C) @ Q.T)
    return w.reshape(-1)


def phi_matrices(X, upto: int, dps: int = 50):
    """[phi_0(X), ..., phi_upto(X)] for a small square X (mpmath exponential of a block matrix)."""
    import mpmath as mp

    X = np.asarray(X, dtype=np.float64)
    k = X.shape[0]
    B = upto + 1
    with mp.workdps(dps):
        Big = mp.zeros(k * B, k * B)
        for a in range(k):
            for b in range(k):
                Big[a, b] = X[a, b]
        for q in range(B - 1):
            for a in range(k):
                Big[q * k + a, (q + 1) * k + a] = 1
        E = mp.expm(Big)
        out = []
        for q in range(B):
            out.append(np.array([[float(E[a, q * k + b]) for b in range(k)] for a in range(k)]))
    return out


def low_rank_comb(U, M, V, t):
    """sum_j phi_j(tA) v_j for A = U M U^T (alpha = 1): sum_j v_j/j! + U (t sum_j phi_{j+1}(tM) W^T v_j),
    W = U M^T (the closed form of the paper's third experiment)."""
    p = V.shape[0] - 1
    W = U @ np.asarray(M).T
    ph = phi_matrices(float(t) * np.asarray(M), p + 1)
    out = np.zeros(U.shape[0])
    inner = np.zeros(U.shape[1])
    for j in range(p + 1):
        out += V[j] / math.factorial(j)
        inner += ph[j + 1] @ (W.T @ V[j])
    return out + U @ (float(t) * inner)


def phi_matrices_ld(X, upto: int):
    """[phi_0(X), ..., phi_upto(X)] for a small square X from the long-double exponential of the same
    block matrix as phi_matrices (no mpmath: usable where only numpy is installed)."""
    X = np.asarray(X, dtype=np.float64)
    k = X.shape[0]
    B = upto + 1
    Big = np.zeros((k * B, k * B), dtype=np.longdouble)
    Big[:k, :k] = X
    for q in range(B - 1):
        for a in range(k):
            Big[q * k + a, (q + 1) * k + a] = 1
    E = expm_longdouble(Big)
    return [E[:k, q * k:(q + 1) * k] for q in range(B)]


def low_rank_comb_ld(U, W, M, V, t, alpha=1.0):
    """sum_j alpha^j phi_j(tA) v_j for A = U W^T with W = U M^T:
    sum_j alpha^j v_j/j! + U (t sum_j alpha^j phi_{j+1}(tM) W^T v_j), in long double."""
    p = V.shape[0] - 1
    ph = phi_matrices_ld(float(t) * np.asarray(M), p + 1)
    Ul = np.asarray(U, dtype=np.longdouble)
    Wl = np.asarray(W, dtype=np.longdouble)
    Vl = np.asarray(V, dtype=np.longdouble)
    a = np.longdouble(alpha)
    out = np.zeros(U.shape[0], dtype=np.longdouble)
    inner = np.zeros(U.shape[1], dtype=np.longdouble)
    for j in range(p + 1):
        out += a**j * Vl[j] / math.factorial(j)
        inner += a**j * (ph[j + 1] @ (Wl.T @ Vl[j]))
    return (out + Ul @ (np.longdouble(t) * inner)).astype(np.float64)
