"""Seeded synthetic inputs: sparse operators A (CSR) and the vectors v_j.

This module holds no arithmetic of the phi-combination method itself; it only builds inputs.
Both the CUDA path and the CPU oracle are fed from here, so it must stay free of the method.

Operators
  * ``laplacian_2d``           -- 5-point Dirichlet Laplacian on an nx x ny interior grid, h = 1/(nx+1),
                                  values (-4, 1, 1, 1, 1)/h^2.
  * ``convection_diffusion``   -- Delta_h - b * sum_d D^-_d (first-order upwind, velocity (b,..,b)),
                                  Dirichlet, h = 1/(nx+1), on a 2-D or 3-D grid; nonnormal for b > 0.
  * ``cheb_laplacian``         -- dense Chebyshev spectral Dirichlet Laplacian on [0, L] (the operator of
                                  the paper's second experiment, Section 5), stored as dense CSR.
  * ``low_rank_dct``           -- A = U M U^T with U the first k orthonormal DCT-II columns (the paper's
                                  third experiment, Section 5), materialised densely for small n.
  * ``diagonal``               -- diagonal CSR.
Vectors
  * ``random_vectors(p, n, seed)`` -- (p+1, n) array, i.i.d. N(0,1) from numpy's PCG64 with ``seed``.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class CSR:
    """CSR matrix with int32 indices; ``values`` is float64 unless converted."""

    n: int
    rowptr: np.ndarray
    colidx: np.ndarray
    values: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.colidx.size)

    def to_dense(self) -> np.ndarray:
        A = np.zeros((self.n, self.n), dtype=np.float64)
        for i in range(self.n):
            lo, hi = self.rowptr[i], self.rowptr[i + 1]
            A[i, self.colidx[lo:hi]] += self.values[lo:hi]
        return A

    def to_scipy(self):
        import scipy.sparse as sp

        return sp.csr_matrix((self.values.astype(np.float64), self.colidx, self.rowptr), shape=(self.n, self.n))

    def scaled(self, c: float) -> "CSR":
        return CSR(self.n, self.rowptr, self.colidx, self.values * c)

    def astype(self, dtype) -> "CSR":
        return CSR(self.n, self.rowptr, self.colidx, self.values.astype(dtype))


def from_scipy(M) -> CSR:
    M = M.tocsr()
    M.sort_indices()
    return CSR(int(M.shape[0]), M.indptr.astype(np.int32), M.indices.astype(np.int32),
               M.data.astype(np.float64))


def dense_to_csr(Ad: np.ndarray, keep_zeros: bool = False) -> CSR:
    Ad = np.asarray(Ad, dtype=np.float64)
    n = Ad.shape[0]
    if keep_zeros:
        rowptr = (np.arange(n + 1, dtype=np.int64) * n).astype(np.int32)
        colidx = np.tile(np.arange(n, dtype=np.int32), n)
        return CSR(n, rowptr, colidx, Ad.reshape(-1).copy())
    import scipy.sparse as sp

    return from_scipy(sp.csr_matrix(Ad))


def diagonal(d) -> CSR:
    d = np.asarray(d, dtype=np.float64)
    n = d.size
    return CSR(n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), d.copy())


def _grid_operator(shape, coeff_center, coeff_minus, coeff_plus) -> CSR:
    """Constant-coefficient stencil on a Dirichlet grid (x fastest).  coeff_minus[d] couples to
    the neighbour at -1 along axis d, coeff_plus[d] to +1; rows keep ascending column order."""
    shape = tuple(int(s) for s in shape)
    dim = len(shape)
    n = int(np.prod(shape))
    idx = np.arange(n, dtype=np.int64)
    coords = []
    rem = idx.copy()
    for d in range(dim):
        coords.append(rem % shape[d])
        rem //= shape[d]
    strides = [int(np.prod(shape[:d])) for d in range(dim)]
    rows, cols, vals = [idx], [idx], [np.full(n, coeff_center, dtype=np.float64)]
    for d in range(dim):
        m = coords[d] > 0
        rows.append(idx[m]); cols.append(idx[m] - strides[d]); vals.append(np.full(int(m.sum()), coeff_minus[d]))
        m = coords[d] < shape[d] - 1
        rows.append(idx[m]); cols.append(idx[m] + strides[d]); vals.append(np.full(int(m.sum()), coeff_plus[d]))
    rows = np.concatenate(rows); cols = np.concatenate(cols); vals = np.concatenate(vals)
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    return CSR(n, rowptr.astype(np.int32), cols.astype(np.int32), vals.astype(np.float64))


def graph_operator(n: int, degree: int, seed: int, hubs: int = 0, hub_degree: int = 0) -> CSR:
    """A = -(L + I) for the weighted Laplacian L = D - W of a random graph on n nodes: degree // 2
    random permutations join i to perm(i), and `hubs` nodes are joined to hub_degree random nodes each;
    weights U(0.5, 1.5), symmetric.  A is symmetric negative definite (eigenvalues in [-1 - 2 max
    weighted degree, -1]); its rows are near-uniform in length (degree + 1) except at the hubs, and its
    stored diagonals are scattered."""
    import scipy.sparse as sp

    rng = np.random.default_rng(seed)
    src, dst = [], []
    for _ in range(degree // 2):
        src.append(np.arange(n)); dst.append(rng.permutation(n))
    for h in rng.choice(n, size=hubs, replace=False) if hubs else []:
        src.append(np.full(hub_degree, h)); dst.append(rng.choice(n, size=hub_degree, replace=False))
    src = np.concatenate(src) if src else np.zeros(0, dtype=np.int64)
    dst = np.concatenate(dst) if dst else np.zeros(0, dtype=np.int64)
    keep = src != dst
    src, dst = src[keep], dst[keep]
    w = rng.uniform(0.5, 1.5, size=src.size)
    Wm = sp.coo_matrix((w, (src, dst)), shape=(n, n)).tocsr()
    Wm = Wm + Wm.T
    L = sp.diags(np.asarray(Wm.sum(axis=1)).ravel()) - Wm
    return from_scipy(-(L + sp.identity(n)))


def laplacian_2d(nx: int, ny: int | None = None) -> CSR:
    ny = nx if ny is None else ny
    h = 1.0 / (nx + 1)
    c = 1.0 / (h * h)
    return _grid_operator((nx, ny), -4.0 * c, [c, c], [c, c])


def laplacian_3d(nx: int) -> CSR:
    h = 1.0 / (nx + 1)
    c = 1.0 / (h * h)
    return _grid_operator((nx, nx, nx), -6.0 * c, [c] * 3, [c] * 3)


def convection_diffusion(nx: int, dim: int, peclet: float) -> CSR:
    """A = Delta_h - b (D^-_1 + ... + D^-_dim), b = peclet (eps = 1, unit box), first-order upwind."""
    h = 1.0 / (nx + 1)
    c = 1.0 / (h * h)
    b = float(peclet) / h
    return _grid_operator((nx,) * dim, -2.0 * dim * c - dim * b, [c + b] * dim, [c] * dim)


def cheb_laplacian(N: int = 100, L: float = 2.0) -> np.ndarray:
    """Dense (N-1) x (N-1) Chebyshev collocation Laplacian on [0, L] with homogeneous Dirichlet
    conditions: the squared differentiation matrix on the Chebyshev points, boundary rows and
    columns removed (second experiment of the paper, Section 5)."""
    j = np.arange(N + 1)
    x = (np.cos(np.pi * j / N) + 1.0) * (L / 2.0)
    c = np.where((j == 0) | (j == N), 2.0, 1.0) * (-1.0) ** j
    dX = x[:, None] - x[None, :]
    D = np.outer(c, 1.0 / c) / (dX + np.eye(N + 1))
    D = D - np.diag(D.sum(axis=1))
    A = (2.0 / L) ** 2 * (D @ D)
    return A[1:N, 1:N].copy()


def dct_basis(n: int, k: int) -> np.ndarray:
    """First k columns of the orthonormal DCT-II matrix (third experiment, Section 5)."""
    i = np.arange(n)[:, None]
    q = np.arange(k)[None, :]
    a = np.where(q == 0, 1.0 / np.sqrt(2.0), 1.0)
    return np.sqrt(2.0 / n) * a * np.cos(np.pi * (i + 0.5) * q / n)


def low_rank_dct(n: int, M: np.ndarray):
    """A = U W^T with W = U M^T, i.e. A = U M U^T.  Returns (A dense, U)."""
    M = np.asarray(M, dtype=np.float64)
    U = dct_basis(n, M.shape[0])
    W = U @ M.T
    return U @ W.T, U


def random_vectors(p: int, n: int, seed: int) -> np.ndarray:
    """(p+1, n) float64, row j = v_j ~ N(0, 1) i.i.d. (numpy PCG64, ``seed``)."""
    return np.random.default_rng(int(seed)).standard_normal((p + 1, int(n)))


# --------------------------------------------------------------------------------------
# Named workloads (sizes and parameters of the benchmark configurations)
# --------------------------------------------------------------------------------------

def workload_laplacian_32():
    """2-D 5-point Dirichlet Laplacian, 32 x 32 grid (n = 1024), p = 3, r = 1, t = 1e-3, alpha = 1,
    tol = 2^-53, v_0..v_3 from seed 1."""
    A = laplacian_2d(32)
    return dict(name="laplace2d-32x32-p3-r1", A=A, V=random_vectors(3, A.n, 1), t=np.array([1e-3]),
                alpha=np.array([1.0]), tol=2.0**-53)


def workload_convdiff3d_64(h: float):
    """expRK4s6-shaped block: 3-D 7-point upwind convection-diffusion on 64^3 (n = 262144),
    Peclet 10; p = 3, r = 2, t = (h/2, h/3), alpha = (1/2, 1/3) (the stage pair c3, c4 of
    expRK4s6 with the scheme weights folded into v_j), tol = 2^-53, v_j from seed 2."""
    A = convection_diffusion(64, 3, 10.0)
    return dict(name=f"convdiff3d-64^3-Pe10-p3-r2-h{h:g}", A=A, V=random_vectors(3, A.n, 2),
                t=np.array([h / 2.0, h / 3.0]), alpha=np.array([0.5, 1.0 / 3.0]), tol=2.0**-53)


def workload_advdiff2d_1024(h: float, tol: float):
    """2-D upwind advection-diffusion on 1024^2 (n = 1,048,576), Peclet 1e3; p = 4, r = 4,
    t = (0.25, 0.5, 0.75, 1) h, alpha = 1, v_j from seed 3."""
    A = convection_diffusion(1024, 2, 1e3)
    return dict(name=f"advdiff2d-1024^2-Pe1e3-p4-r4-h{h:g}", A=A, V=random_vectors(4, A.n, 3),
                t=np.array([0.25, 0.5, 0.75, 1.0]) * h, alpha=np.ones(4), tol=tol)


# ---- many uneven instances (batched launches) -------------------------------------------------------
def shifted_laplacian(shape, shift: np.ndarray) -> CSR:
    """Dirichlet Laplacian on a grid of the given shape (h_d = 1/(shape_d + 1) per axis, scaled by
    1/h_d^2) plus diag(shift)."""
    cd = [float(s + 1) ** 2 for s in shape]
    A = _grid_operator(shape, -2.0 * sum(cd), cd, cd)
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    diag = A.colidx == rows
    vals = A.values.copy()
    vals[diag] += np.asarray(shift, dtype=np.float64)[rows[diag]]
    return CSR(A.n, A.rowptr, A.colidx, vals)


def batch_instance(seed: int, i: int, n_lo: int = 1000, n_hi: int = 256000, precision: str = "mixed") -> dict:
    """Instance i of the batching workload: n log-uniform in [n_lo, n_hi] (2-D or 3-D grid, equally
    likely), a Dirichlet Laplacian plus diagonal shifts U[-10, 0], p in 1..4, r in 1..3, v_j ~ N(0, 1),
    t_i = tau (i / r) / rho with rho = 4 sum_d 1/h_d^2 + 10 (a Gershgorin bound of |A|) and tau
    log-uniform in [1, 100], alpha_i ~ U[0.5, 1.5].  precision "mixed" draws FP64 (tol 2^-53) or FP32
    (tol 2^-24) with equal odds; "f64" / "f32" fix it."""
    rng = np.random.default_rng([int(seed), int(i)])
    n_target = float(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi))))
    dim = int(rng.integers(2, 4))
    if dim == 2:
        nx = max(2, int(round(np.sqrt(n_target))))
        shape = (nx, max(2, int(round(n_target / nx))))
    else:
        nx = max(2, int(round(n_target ** (1.0 / 3.0))))
        shape = (nx, nx, max(2, int(round(n_target / (nx * nx)))))
    n = int(np.prod(shape))
    shift = rng.uniform(-10.0, 0.0, size=n)
    p = int(rng.integers(1, 5))
    r = int(rng.integers(1, 4))
    rho = 4.0 * sum(float(s + 1) ** 2 for s in shape) + 10.0
    tau = float(np.exp(rng.uniform(0.0, np.log(100.0))))
    t = tau * np.arange(1, r + 1) / r / rho
    alpha = rng.uniform(0.5, 1.5, size=r)
    f32 = bool(rng.integers(0, 2)) if precision == "mixed" else precision == "f32"
    V = rng.standard_normal((p + 1, n))
    return dict(name=f"batch{seed}-{i}", A=shifted_laplacian(shape, shift), V=V, t=t, alpha=alpha, p=p, r=r,
                prec="f32" if f32 else "f64", tol=2.0**-24 if f32 else 2.0**-53, shape=shape)


def workload_batch(count: int = 512, seed: int = 4, precision: str = "mixed", n_lo: int = 1000,
                   n_hi: int = 256000) -> list:
    """The batching workload: `count` independent instances (see batch_instance)."""
    return [batch_instance(seed, i, n_lo, n_hi, precision) for i in range(count)]


# ---- the paper's ADR problem (Section 6, fourth experiment) ----------------------------------------
ADR_EPS, ADR_ALPHA, ADR_GAMMA = 1e-3, -0.5, 1000.0


def adr_operator(N: int = 100, eps: float = ADR_EPS, alpha: float = ADR_ALPHA) -> CSR:
    """A = eps Laplacian - alpha (d/dx + d/dy) on [0,1]^2 with N nodes per direction: nodes
    x_i = i / N, i = 0..N-1 (spacing 1/N); homogeneous Neumann at x = 0 and y = 0 (ghost value
    u_{-1} = u_1), homogeneous Dirichlet at x = 1 and y = 1 (node N is the boundary, u = 0); second-order
    central differences for both terms; x fastest.  n = N^2 (10^4 for N = 100)."""
    import scipy.sparse as sp

    dx = 1.0 / N
    main = np.full(N, -2.0 / dx**2)
    lo = np.full(N - 1, 1.0 / dx**2)
    up = np.full(N - 1, 1.0 / dx**2)
    up[0] = 2.0 / dx**2  # Neumann ghost at node 0: u_{-1} = u_1
    L1 = sp.diags([lo, main, up], [-1, 0, 1], format="csr")
    dlo = np.full(N - 1, -1.0 / (2 * dx))
    dup = np.full(N - 1, 1.0 / (2 * dx))
    dup[0] = 0.0  # (u_1 - u_{-1}) / (2 dx) = 0 at the Neumann node
    D1 = sp.diags([dlo, dup], [-1, 1], format="csr")
    I = sp.identity(N, format="csr")
    A = eps * (sp.kron(I, L1) + sp.kron(L1, I)) - alpha * (sp.kron(I, D1) + sp.kron(D1, I))
    A = sp.csr_matrix(A)
    A.sort_indices()
    return from_scipy(A)


def adr_initial(N: int = 100) -> np.ndarray:
    """u(0, x, y) = 256 x^2 y^2 (1-x)^2 (1-y)^2 on the nodes of adr_operator."""
    x = np.arange(N) / N
    X, Y = np.meshgrid(x, x, indexing="xy")
    return (256.0 * X**2 * Y**2 * (1 - X) ** 2 * (1 - Y) ** 2).ravel()
