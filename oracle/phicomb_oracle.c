/*
 * Oracle for the phi-combination method of Al-Mohy, "Computing Linear Combinations of
 * phi-Function Actions for Exponential Integrators" (arXiv 2509.26475).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, FP64 CPU restatement of the
 * paper's Algorithm 1 (selection of the scaling s and shift xi), Algorithm 2 (one
 * combination) and Algorithm 3 (r combinations in block form).  It is used by the test
 * suite, by the smoke check and by the timed CPU baseline of the benchmark, and by
 * nothing else.  It shares no code with the CUDA library.
 *
 * Conventions
 *   - A is CSR: rowptr[n+1], colidx[nnz] (int32), val[nnz] (double).
 *   - A block X with w columns is stored column by column: X[c*n + i] is row i of column c,
 *     matching the paper's matrix notation (columns are vectors).
 *   - Every loop follows the order in which the paper states the step; the only library
 *     routines used are libm's exp, log, sqrt, pow, lgamma, ceil.
 *   - Built with -ffp-contract=off so that no multiply-add is fused: results are the same
 *     on x86-64 and aarch64.
 *   - The only parallelism is an optional OpenMP split of the rows of a sparse product;
 *     every row is computed by one thread in CSR order, so results do not depend on the
 *     thread count.
 *
 * Readings of passages that are ambiguous in the paper (each is also listed in the design
 * notes of the repository):
 *   R1  Algorithm 3 forms the shifted nilpotent factor without a division by s; it is
 *       divided by s as in Algorithm 2:  Jsh = (J (x) Delta - xi I (x) T) / s.
 *   R2  The recovery recurrence uses S <- S*Jt before the refresh of F (exponent k), as the
 *       algorithms state.
 *   R4  ||X||_inf of an n x w block is the matrix infinity norm: max over rows of the sum of
 *       |X(i,c)| over all w columns (jointly over the r combinations).
 *   R5  The truncation test is applied after every term, with c1 = infinity on entry.
 *   R6  Each Taylor loop is capped at max_terms terms (default 10*61); hitting the cap
 *       returns ORC_TERM_CAP.
 *   R8  2-norms use max-abs scaling: ||x|| = M*sqrt(sum (x_i/M)^2), log||x|| = log M + log(sum)/2.
 *   R9  r = 0 (A v underflows) gives xi = 0, s = 1.  When r - j_r <= 0, j_r = max(0, r-1).
 *   R10 Brent's minimiser (Brent 1973, ch. 5): golden section plus parabolic steps,
 *       tolerance eps*|x| + tabs with eps = sqrt(2^-52), tabs = 1e-8*s0, at most
 *       max_evals evaluations.
 *   R12 s_int = max(1, ceil(s*max|t_i|)).
 *   R13 real arithmetic only; xi is searched on the real bracket [-sqrt(n) s0, sqrt(n) s0].
 *   R14 p = 0 carries only the first block column of F (see orc_solve).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <float.h>

#define ORC_OK 0
#define ORC_INVALID_ARG 1
#define ORC_NONFINITE 2
#define ORC_TERM_CAP 3
#define ORC_NO_MEMORY 7

#define ORC_FLAG_NO_V0 1u /* v0 omitted: w_i = alpha_i * sum_{j>=1} alpha_i^{j-1} phi_j(t_i A) v_j */

#define ORC_MAX_M 256

typedef struct {
  int64_t n, nnz;
  const int32_t* rowptr;
  const int32_t* colidx;
  const double* val;
} orc_csr;

typedef struct {
  double xi;      /* optimal shift xi* */
  double s;       /* scaling parameter s (real, > 0) */
  double s0;      /* preliminary scale from the power basis */
  double f_star;  /* objective value f(xi*) */
  int32_t r;      /* last accepted power index */
  int32_t evals;  /* objective evaluations spent by the minimiser */
  double L[ORC_MAX_M + 1]; /* log ||A^k v||_2, k = 0..r (entries past r undefined) */
} orc_select_out;

typedef struct {
  int32_t status;
  int32_t s_int;
  int32_t series_terms;    /* value of k when the S-series loop stops */
  int32_t max_inner_terms; /* largest k over the recovery steps */
  int64_t recovery_terms;  /* total inner terms over the s_int - 1 recovery steps */
  int64_t spmm_count;      /* sparse products with a block (one per term, plus the first-block recovery) */
} orc_stats;

/* ------------------------------------------------------------------------------------ */
/* Basic blocks                                                                         */
/* ------------------------------------------------------------------------------------ */

/* Y(:,c) = A X(:,c) for c = 0..w-1 (columns of length n). */
static void csr_times_block(const orc_csr* A, const double* X, int w, double* Y) {
  const int64_t n = A->n;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (int64_t i = 0; i < n; ++i) {
    for (int c = 0; c < w; ++c) {
      double acc = 0.0;
      for (int32_t q = A->rowptr[i]; q < A->rowptr[i + 1]; ++q) acc += A->val[q] * X[(int64_t)c * n + A->colidx[q]];
      Y[(int64_t)c * n + i] = acc;
    }
  }
}

/* Matrix infinity norm of an n x w block: max_i sum_c |X(i,c)|  (reading R4). */
static double norm_inf(const double* X, int64_t n, int w) {
  double best = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double rs = 0.0;
    for (int c = 0; c < w; ++c) rs += fabs(X[(int64_t)c * n + i]);
    if (!(rs <= best)) best = rs; /* propagates NaN */
  }
  return best;
}

/* log of the 2-norm with max-abs scaling (reading R8).  Returns -inf for a zero vector. */
static double log_norm2(const double* x, int64_t n) {
  double M = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double a = fabs(x[i]);
    if (!(a <= M)) M = a;
  }
  if (M == 0.0) return -INFINITY;
  if (!isfinite(M)) return M;
  double ssq = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double y = x[i] / M;
    ssq += y * y;
  }
  return log(M) + 0.5 * log(ssq);
}

static double norm2(const double* x, int64_t n) {
  double l = log_norm2(x, n);
  return isinf(l) && l < 0 ? 0.0 : exp(l);
}

/* C = X * M for an n x w block X and a dense w x w matrix M (row-major M[a*w+b]). */
static void block_times_small(const double* X, int64_t n, int w, const double* M, double* C) {
  for (int b = 0; b < w; ++b) {
    double* Cb = C + (int64_t)b * n;
    for (int64_t i = 0; i < n; ++i) Cb[i] = 0.0;
    for (int a = 0; a < w; ++a) {
      double m = M[a * w + b];
      if (m == 0.0) continue;
      const double* Xa = X + (int64_t)a * n;
      for (int64_t i = 0; i < n; ++i) Cb[i] += Xa[i] * m;
    }
  }
}

/* ------------------------------------------------------------------------------------ */
/* Counter-based generator for the unit vector of Algorithm 1 (reading R7).             */
/* splitmix64 (Steele, Lea and Flood 2014): state_i = seed + (i+1)*0x9E3779B97F4A7C15,   */
/* then the published three-step finaliser; u = (z >> 11) * 2^-53, x = 2u - 1.          */
/* ------------------------------------------------------------------------------------ */
static uint64_t orc_splitmix64_at(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

void orc_unit_vector(int64_t n, uint64_t seed, double* v) {
  for (int64_t i = 0; i < n; ++i) {
    double u = (double)(orc_splitmix64_at(seed, (uint64_t)i) >> 11) * 0x1.0p-53;
    v[i] = 2.0 * u - 1.0;
  }
}

/* ------------------------------------------------------------------------------------ */
/* Algorithm 1: power basis, preliminary scale s0, objective f(xi), Brent, s.            */
/* ------------------------------------------------------------------------------------ */

/* Safe power basis, its normalisation and extension to degree m (Algorithm 1, steps
 * "build safe powers" through "normalize and extend").  V is n x (m+1), column k = V_k.
 * On return *r_out is the last accepted index and *s0_out the preliminary scale.
 * Returns ORC_OK, or ORC_INVALID_ARG. */
int orc_power_basis(const orc_csr* A, int m, double delta, const double* v, double* V, double* L,
                    int* r_out, double* s0_out) {
  const int64_t n = A->n;
  if (m < 1 || m > ORC_MAX_M || n < 1) return ORC_INVALID_ARG;
  const double g_max = delta * log(DBL_MAX);
  const double g_min = delta * log(DBL_MIN);
  /* l_j = log binom(m, j); l_max = max_j l_j */
  double l_max = -INFINITY;
  for (int j = 0; j <= m; ++j) {
    double lj = lgamma(m + 1.0) - lgamma(j + 1.0) - lgamma(m - j + 1.0);
    if (lj > l_max) l_max = lj;
  }
  /* V_0 = v / ||v||_2 */
  double nv = norm2(v, n);
  if (!(nv > 0.0) || !isfinite(nv)) return ORC_INVALID_ARG;
  for (int64_t i = 0; i < n; ++i) V[i] = v[i] / nv;
  L[0] = log_norm2(V, n);
  int r = 0;
  double* W = (double*)malloc(sizeof(double) * (size_t)n);
  if (!W) return ORC_NO_MEMORY;
  for (int k = 1; k <= m; ++k) {
    csr_times_block(A, V + (int64_t)(k - 1) * n, 1, W); /* W_k = A V_{k-1} */
    double Lk = log_norm2(W, n);                         /* L_k = log ||W_k||_2 */
    if (Lk + 0.5 * log(k + 1.0) + l_max > g_max || Lk < g_min || isnan(Lk)) break;
    memcpy(V + (int64_t)k * n, W, sizeof(double) * (size_t)n); /* V_k = W_k */
    L[k] = Lk;
    r = k;
  }
  *r_out = r;
  if (r == 0) { /* reading R9: nothing accepted */
    free(W);
    *s0_out = 0.0;
    return ORC_OK;
  }
  int jr = r - 5 > 2 ? r - 5 : 2;
  if (r - jr <= 0) jr = r - 1 > 0 ? r - 1 : 0;
  double acc = 0.0;
  for (int j = jr; j <= r - 1; ++j) acc += L[j + 1] - L[j];
  double s0 = exp(acc / (double)(r - jr)); /* geometric mean of the last growth factors */
  for (int j = 1; j <= r; ++j) {
    double sc = pow(s0, -(double)j);
    double* Vj = V + (int64_t)j * n;
    for (int64_t i = 0; i < n; ++i) Vj[i] *= sc;
  }
  for (int k = r + 1; k <= m; ++k) { /* V_k = s0^{-1} A V_{k-1} */
    double* Vk = V + (int64_t)k * n;
    csr_times_block(A, V + (int64_t)(k - 1) * n, 1, Vk);
    for (int64_t i = 0; i < n; ++i) Vk[i] /= s0;
  }
  free(W);
  *s0_out = s0;
  return ORC_OK;
}

/* Objective f(xi) = || V (b .* p(xi)) ||_2^(1/m),  z = -xi/s0,  p = [z^m..z,1],
 * b = [binom(m,0)..binom(m,m)].  Column V_k meets b_k z^(m-k).  y is scratch of length n. */
double orc_objective(const double* V, int64_t n, int m, double s0, double xi, double* y) {
  double z = -xi / s0;
  for (int64_t i = 0; i < n; ++i) y[i] = 0.0;
  double binom = 1.0; /* binom(m, k), updated multiplicatively */
  for (int k = 0; k <= m; ++k) {
    if (k > 0) binom = binom * (double)(m - k + 1) / (double)k;
    double coef = binom * pow(z, (double)(m - k));
    const double* Vk = V + (int64_t)k * n;
    for (int64_t i = 0; i < n; ++i) y[i] += coef * Vk[i];
  }
  double l = log_norm2(y, n);
  if (isinf(l) && l < 0) return 0.0;
  return exp(l / (double)m);
}

typedef struct {
  const double* V;
  int64_t n;
  int m;
  double s0;
  double* y;
} orc_obj_ctx;

static double obj_eval(void* ctx, double xi) {
  orc_obj_ctx* c = (orc_obj_ctx*)ctx;
  return orc_objective(c->V, c->n, c->m, c->s0, xi, c->y);
}

typedef double (*orc_fn)(void* ctx, double x);

/* Brent's derivative-free minimiser on [a, b] (Brent 1973, ch. 5; reading R10).
 * Keeps the best point x, the second best w and the previous w (v); tries a parabola
 * through them and falls back to a golden-section step into the larger part.
 * *evals counts the function evaluations. */
static double brent_min(orc_fn fn, void* ctx, double a, double b, double tabs, int max_evals, double* fmin,
                        int* evals) {
  const double gold = 0.5 * (3.0 - sqrt(5.0));
  const double eps = sqrt(0x1.0p-52);
  double x = a + gold * (b - a);
  double w = x, v = x;
  double fx = fn(ctx, x);
  int ne = 1;
  double fw = fx, fv = fx;
  double d = 0.0, e = 0.0;
  while (ne < max_evals) {
    double mid = 0.5 * (a + b);
    double tol1 = eps * fabs(x) + tabs / 3.0;
    double tol2 = 2.0 * tol1;
    if (fabs(x - mid) <= tol2 - 0.5 * (b - a)) break; /* bracket small enough */
    int golden = 1;
    if (fabs(e) > tol1) {
      /* parabola through (x,fx), (w,fw), (v,fv): step num/den from x */
      double t1 = (x - w) * (fx - fv);
      double t2 = (x - v) * (fx - fw);
      double num = (x - v) * t2 - (x - w) * t1;
      double den = 2.0 * (t2 - t1);
      if (den > 0.0) num = -num; else den = -den;
      double e_prev = e;
      e = d;
      if (fabs(num) < fabs(0.5 * den * e_prev) && num > den * (a - x) && num < den * (b - x)) {
        d = num / den;
        double u = x + d;
        if (u - a < tol2 || b - u < tol2) d = (mid >= x) ? tol1 : -tol1;
        golden = 0;
      }
    }
    if (golden) {
      e = (x >= mid) ? a - x : b - x;
      d = gold * e;
    }
    double u = (fabs(d) >= tol1) ? x + d : x + (d > 0.0 ? tol1 : -tol1);
    double fu = fn(ctx, u);
    ne++;
    if (fu <= fx) {
      if (u >= x) a = x; else b = x;
      v = w; fv = fw;
      w = x; fw = fx;
      x = u; fx = fu;
    } else {
      if (u < x) a = u; else b = u;
      if (fu <= fw || w == x) {
        v = w; fv = fw;
        w = u; fw = fu;
      } else if (fu <= fv || v == x || v == w) {
        v = u; fv = fu;
      }
    }
  }
  *fmin = fx;
  *evals = ne;
  return x;
}

/* The minimiser on a caller-supplied function (used to pin it on functions with known minima). */
double orc_minimize(orc_fn fn, void* ctx, double a, double b, double tabs, int max_evals, double* fmin, int* evals) {
  return brent_min(fn, ctx, a, b, tabs, max_evals, fmin, evals);
}

/* Algorithm 1.  v may be NULL: then v is drawn with orc_unit_vector(n, seed).
 * V_work must hold n*(m+1) doubles (the basis is left there for inspection). */
int orc_select(const orc_csr* A, int m, double tol, double delta, const double* v, uint64_t seed, int max_evals,
               double* V_work, orc_select_out* out) {
  const int64_t n = A->n;
  if (!A || !out || m < 1 || m > ORC_MAX_M || !(tol > 0.0) || !(delta > 0.0) || n < 1) return ORC_INVALID_ARG;
  double* vv = NULL;
  if (!v) {
    vv = (double*)malloc(sizeof(double) * (size_t)n);
    if (!vv) return ORC_NO_MEMORY;
    orc_unit_vector(n, seed, vv);
    v = vv;
  }
  memset(out, 0, sizeof(*out));
  int r = 0;
  double s0 = 0.0;
  int st = orc_power_basis(A, m, delta, v, V_work, out->L, &r, &s0);
  free(vv);
  if (st != ORC_OK) return st;
  out->r = r;
  out->s0 = s0;
  if (r == 0) { /* reading R9 */
    out->xi = 0.0;
    out->s = 1.0;
    out->f_star = 0.0;
    return ORC_OK;
  }
  double* y = (double*)malloc(sizeof(double) * (size_t)n);
  if (!y) return ORC_NO_MEMORY;
  orc_obj_ctx c = {V_work, n, m, s0, y};
  double half = sqrt((double)n) * s0; /* bracket [-sqrt(n) s0, sqrt(n) s0] */
  double fstar = 0.0;
  int evals = 0;
  double xi = brent_min(obj_eval, &c, -half, half, 1e-8 * s0, max_evals, &fstar, &evals);
  free(y);
  double lg = (log(tol) + lgamma(m + 1.0)) / (double)m; /* log (tol m!)^(1/m) */
  out->xi = xi;
  out->f_star = fstar;
  out->evals = evals;
  out->s = s0 * fstar / exp(lg);
  if (!isfinite(out->s) || !isfinite(out->xi)) return ORC_NONFINITE;
  return ORC_OK;
}

/* Evaluate f at a given xi on the basis of A (for comparing another implementation's xi*). */
int orc_objective_at(const orc_csr* A, int m, double delta, const double* v, const double* xis, int nxi, double* f_out,
                     double* s0_out, int* r_out) {
  const int64_t n = A->n;
  double* V = (double*)malloc(sizeof(double) * (size_t)n * (size_t)(m + 1));
  double* L = (double*)malloc(sizeof(double) * (size_t)(m + 1));
  double* y = (double*)malloc(sizeof(double) * (size_t)n);
  if (!V || !L || !y) { free(V); free(L); free(y); return ORC_NO_MEMORY; }
  int r = 0;
  double s0 = 0.0;
  int st = orc_power_basis(A, m, delta, v, V, L, &r, &s0);
  if (st == ORC_OK) {
    for (int q = 0; q < nxi; ++q) f_out[q] = r > 0 ? orc_objective(V, n, m, s0, xis[q], y) : 0.0;
    *s0_out = s0;
    *r_out = r;
  }
  free(V); free(L); free(y);
  return st;
}

/* ------------------------------------------------------------------------------------ */
/* Algorithm 3 (block form; r combinations).                                            */
/* ------------------------------------------------------------------------------------ */

/* Vin is (p+1) x n: vector v_j at Vin + j*n.  t and alpha have r entries.  s and xi come
 * from Algorithm 1.  W receives r vectors: w_i at W + i*n.  max_terms <= 0 selects 610. */
int orc_solve(const orc_csr* A, int p, int r, const double* Vin, const double* t, const double* alpha, double tol,
              double s, double xi, unsigned flags, int max_terms, double* W, orc_stats* st) {
  const int64_t n = A->n;
  if (!A || !Vin || !t || !alpha || !W || p < 0 || r < 1 || n < 1 || !(tol > 0.0) || !(s >= 0.0) || !isfinite(xi))
    return ORC_INVALID_ARG;
  if (max_terms <= 0) max_terms = 610;
  orc_stats local;
  if (!st) st = &local;
  memset(st, 0, sizeof(*st));
  const int P = p + 1;     /* columns of V */
  const int w = P * r;     /* columns of the block series */
  const int no_v0 = (flags & ORC_FLAG_NO_V0) != 0;

  /* s <- ceil(s max|t_i|)  (reading R12) */
  double tmax = 0.0;
  for (int i = 0; i < r; ++i) if (fabs(t[i]) > tmax) tmax = fabs(t[i]);
  double sc = ceil(s * tmax);
  if (!(sc >= 1.0)) sc = 1.0;
  if (sc > 2147483647.0) return ORC_INVALID_ARG;
  const int s_int = (int)sc;
  st->s_int = s_int;

  /* mu = exp((xi/s) T) */
  double* mu = (double*)malloc(sizeof(double) * r);
  for (int i = 0; i < r; ++i) mu[i] = exp(xi * t[i] / (double)s_int);

  /* V <- [v0, vp, ..., v1], then V <- V (I_{p+1} kron 1_r^T mu/s): column (b,i) = b*r + i */
  double* Vb = (double*)calloc((size_t)n * w, sizeof(double));
  for (int b = 0; b < P; ++b) {
    const double* src = (b == 0) ? Vin : Vin + (int64_t)(p + 1 - b) * n; /* reordered column b */
    for (int i = 0; i < r; ++i) {
      double f = mu[i] / (double)s_int;
      double* dst = Vb + (int64_t)(b * r + i) * n;
      for (int64_t q = 0; q < n; ++q) dst[q] = (b == 0 && no_v0) ? 0.0 : src[q] * f;
    }
  }

  /* J = [0] (+) J_p(0): J[a][a+1] = 1 for a = 1..p-1.  Kronecker products are w x w. */
  double* JD = (double*)calloc((size_t)w * w, sizeof(double));  /* J kron Delta */
  for (int a = 1; a <= p - 1; ++a)
    for (int i = 0; i < r; ++i) JD[(a * r + i) * w + ((a + 1) * r + i)] = alpha[i];
  /* Jt = exp(J kron Delta / s): the argument is nilpotent, so the series ends after p terms */
  double* Jt = (double*)calloc((size_t)w * w, sizeof(double));
  double* Pw = (double*)calloc((size_t)w * w, sizeof(double));
  double* Tmp = (double*)calloc((size_t)w * w, sizeof(double));
  for (int a = 0; a < w; ++a) Pw[a * w + a] = 1.0;
  for (int a = 0; a < w; ++a) Jt[a * w + a] = 1.0;
  for (int q = 1; q <= p; ++q) {
    /* Pw <- Pw (J kron Delta / s) / q */
    for (int a = 0; a < w; ++a)
      for (int b = 0; b < w; ++b) {
        double acc = 0.0;
        for (int c = 0; c < w; ++c) acc += Pw[a * w + c] * (JD[c * w + b] / (double)s_int);
        Tmp[a * w + b] = acc / (double)q;
      }
    memcpy(Pw, Tmp, sizeof(double) * (size_t)w * w);
    for (int a = 0; a < w * w; ++a) Jt[a] += Pw[a];
  }
  /* Jsh = (J kron Delta - xi I_{p+1} kron T) / s   (reading R1) */
  double* Jsh = (double*)calloc((size_t)w * w, sizeof(double));
  for (int a = 0; a < w; ++a)
    for (int b = 0; b < w; ++b) {
      double v = JD[a * w + b];
      if (a == b) v -= xi * t[a % r];
      Jsh[a * w + b] = v / (double)s_int;
    }

  double* S = (double*)malloc(sizeof(double) * (size_t)n * w);
  double* D = (double*)malloc(sizeof(double) * (size_t)n * w);
  double* Y = (double*)malloc(sizeof(double) * (size_t)n * w);
  double* Vn = (double*)malloc(sizeof(double) * (size_t)n * w);
  memcpy(S, Vb, sizeof(double) * (size_t)n * w);
  memcpy(D, Vb, sizeof(double) * (size_t)n * w);
  int status = ORC_OK;

  /* ---- block series S = sum D_k / k!  with the truncation test ---- */
  int k = 1;
  double sigma = 1.0;
  double c1 = INFINITY, c2 = norm_inf(D, n, w);
  for (;;) {
    const double nS = norm_inf(S, n, w);
    if (!isfinite(c2) || !isfinite(nS)) { status = ORC_NONFINITE; break; } /* a NaN would end the test silently */
    if (!(c1 + c2 > tol * nS)) break;
    if (k >= max_terms) { status = ORC_TERM_CAP; break; }
    k = k + 1;
    c1 = c2;
    sigma = k * sigma;
    block_times_small(Vb, n, w, Jsh, Vn); /* V <- V Jsh */
    memcpy(Vb, Vn, sizeof(double) * (size_t)n * w);
    csr_times_block(A, D, w, Y);           /* A D */
    st->spmm_count++;
    for (int c = 0; c < w; ++c) {          /* D <- (A - xi I) D (I kron T/s) + V */
      double tc = t[c % r] / (double)s_int;
      for (int64_t q = 0; q < n; ++q) {
        int64_t idx = (int64_t)c * n + q;
        D[idx] = (Y[idx] - xi * D[idx]) * tc + Vb[idx];
      }
    }
    c2 = norm_inf(D, n, w) / sigma;
    for (int64_t idx = 0; idx < (int64_t)n * w; ++idx) S[idx] = S[idx] + D[idx] / sigma;
  }
  st->series_terms = k;

  /* ---- F = S(:, [1:r, pr+1:(p+1)r]) ;  F(:,1:r) <- A F(:,1:r) T + v0 1^T ----
   * Reading R14: with p = 0 (only v0 given, the output option e^{tA} v0 of Section 4) both block
   * columns are column block 0, the second copy never reaches the output, and only the first block
   * is carried (its norms alone enter the truncation test). */
  const int wf = (p == 0) ? r : 2 * r;
  double* F = (double*)malloc(sizeof(double) * (size_t)n * wf);
  double* E = (double*)malloc(sizeof(double) * (size_t)n * wf);
  double* Yf = (double*)malloc(sizeof(double) * (size_t)n * wf);
  for (int i = 0; i < r; ++i) {
    memcpy(F + (int64_t)i * n, S + (int64_t)i * n, sizeof(double) * (size_t)n);
    if (p > 0) memcpy(F + (int64_t)(r + i) * n, S + (int64_t)(p * r + i) * n, sizeof(double) * (size_t)n);
  }
  if (status == ORC_OK) {
    csr_times_block(A, F, r, Yf);
    st->spmm_count++;
    for (int i = 0; i < r; ++i)
      for (int64_t q = 0; q < n; ++q)
        F[(int64_t)i * n + q] = Yf[(int64_t)i * n + q] * t[i] + (no_v0 ? 0.0 : Vin[q]);
  }

  /* ---- recovery: s_int - 1 applications of exp(A/s) with the undo factor mu ---- */
  double* Sn = (double*)malloc(sizeof(double) * (size_t)n * w);
  for (int j = 1; j <= s_int - 1 && status == ORC_OK; ++j) {
    memcpy(E, F, sizeof(double) * (size_t)n * wf);
    int kk = 0;
    double d1 = INFINITY, d2 = norm_inf(F, n, wf);
    for (;;) {
      const double nE = norm_inf(E, n, wf);
      if (!isfinite(d2) || !isfinite(nE)) { status = ORC_NONFINITE; break; }
      if (!(d1 + d2 > tol * nE)) break;
      if (kk >= max_terms) { status = ORC_TERM_CAP; break; }
      kk = kk + 1;
      d1 = d2;
      csr_times_block(A, F, wf, Yf); /* F <- (A - xi I) F (I_2 kron T/s) / k */
      st->spmm_count++;
      for (int c = 0; c < wf; ++c) {
        double tc = t[c % r] / (double)s_int;
        for (int64_t q = 0; q < n; ++q) {
          int64_t idx = (int64_t)c * n + q;
          F[idx] = (Yf[idx] - xi * F[idx]) * tc / (double)kk;
        }
      }
      d2 = norm_inf(F, n, wf);
      for (int64_t idx = 0; idx < (int64_t)n * wf; ++idx) E[idx] = E[idx] + F[idx];
    }
    st->recovery_terms += kk;
    if (kk > st->max_inner_terms) st->max_inner_terms = kk;
    if (status != ORC_OK) break;
    for (int c = 0; c < wf; ++c) { /* E <- E (I_2 kron mu) */
      double m_c = mu[c % r];
      for (int64_t q = 0; q < n; ++q) E[(int64_t)c * n + q] *= m_c;
    }
    block_times_small(S, n, w, Jt, Sn); /* S <- S Jt */
    memcpy(S, Sn, sizeof(double) * (size_t)n * w);
    for (int i = 0; i < r; ++i) {       /* F <- E + S(:, [blk 0, blk p]) ; F(:,1:r) <- E(:,1:r) */
      for (int64_t q = 0; q < n; ++q) {
        F[(int64_t)i * n + q] = E[(int64_t)i * n + q];
        if (p > 0) F[(int64_t)(r + i) * n + q] = E[(int64_t)(r + i) * n + q] + S[(int64_t)(p * r + i) * n + q];
      }
    }
  }

  /* ---- w_i = F(:, i) + alpha_i F(:, r+i);  p = 0 returns exp(t_i A) v0 ---- */
  for (int i = 0; i < r; ++i)
    for (int64_t q = 0; q < n; ++q) {
      double f1 = F[(int64_t)i * n + q];
      W[(int64_t)i * n + q] = (p == 0) ? f1 : f1 + alpha[i] * F[(int64_t)(r + i) * n + q];
    }
  st->status = status;
  free(mu); free(Vb); free(JD); free(Jt); free(Pw); free(Tmp); free(Jsh);
  free(S); free(D); free(Y); free(Vn); free(F); free(E); free(Yf); free(Sn);
  return status;
}

/* ------------------------------------------------------------------------------------ */
/* Algorithm 2 (one combination), kept as written for scalar t and alpha.               */
/* ------------------------------------------------------------------------------------ */
int orc_solve_single(const orc_csr* A, int p, const double* Vin, double t, double alpha, double tol, double s,
                     double xi, int max_terms, double* w_out, orc_stats* st) {
  const int64_t n = A->n;
  if (!A || !Vin || !w_out || p < 0 || n < 1 || !(tol > 0.0) || !(s >= 0.0)) return ORC_INVALID_ARG;
  if (max_terms <= 0) max_terms = 610;
  orc_stats local;
  if (!st) st = &local;
  memset(st, 0, sizeof(*st));
  const int P = p + 1;
  double sc = ceil(fabs(t) * s);
  if (!(sc >= 1.0)) sc = 1.0;
  const int s_int = (int)sc;
  st->s_int = s_int;
  const double mu = exp(t * xi / (double)s_int);
  /* J <- alpha J; V <- [v0, vp, ..., v1]; V <- (mu/s) V */
  double* Vb = (double*)malloc(sizeof(double) * (size_t)n * P);
  for (int b = 0; b < P; ++b) {
    const double* src = (b == 0) ? Vin : Vin + (int64_t)(p + 1 - b) * n;
    for (int64_t q = 0; q < n; ++q) Vb[(int64_t)b * n + q] = (mu / (double)s_int) * src[q];
  }
  double* aJ = (double*)calloc((size_t)P * P, sizeof(double));
  for (int a = 1; a <= p - 1; ++a) aJ[a * P + a + 1] = alpha;
  /* Jt = e^{J/s}, J <- (J - t xi I)/s */
  double* Jt = (double*)calloc((size_t)P * P, sizeof(double));
  double* Pw = (double*)calloc((size_t)P * P, sizeof(double));
  double* Tmp = (double*)calloc((size_t)P * P, sizeof(double));
  for (int a = 0; a < P; ++a) { Jt[a * P + a] = 1.0; Pw[a * P + a] = 1.0; }
  for (int q = 1; q <= p; ++q) {
    for (int a = 0; a < P; ++a)
      for (int b = 0; b < P; ++b) {
        double acc = 0.0;
        for (int c = 0; c < P; ++c) acc += Pw[a * P + c] * (aJ[c * P + b] / (double)s_int);
        Tmp[a * P + b] = acc / (double)q;
      }
    memcpy(Pw, Tmp, sizeof(double) * (size_t)P * P);
    for (int a = 0; a < P * P; ++a) Jt[a] += Pw[a];
  }
  double* Js = (double*)calloc((size_t)P * P, sizeof(double));
  for (int a = 0; a < P; ++a)
    for (int b = 0; b < P; ++b) Js[a * P + b] = (aJ[a * P + b] - (a == b ? t * xi : 0.0)) / (double)s_int;
  double* S = (double*)malloc(sizeof(double) * (size_t)n * P);
  double* D = (double*)malloc(sizeof(double) * (size_t)n * P);
  double* Y = (double*)malloc(sizeof(double) * (size_t)n * P);
  double* Vn = (double*)malloc(sizeof(double) * (size_t)n * P);
  memcpy(S, Vb, sizeof(double) * (size_t)n * P);
  memcpy(D, Vb, sizeof(double) * (size_t)n * P);
  int status = ORC_OK;
  int k = 1;
  double sigma = 1.0, c1 = INFINITY, c2 = norm_inf(D, n, P);
  for (;;) {
    const double nS = norm_inf(S, n, P);
    if (!isfinite(c2) || !isfinite(nS)) { status = ORC_NONFINITE; break; }
    if (!(c1 + c2 > tol * nS)) break;
    if (k >= max_terms) { status = ORC_TERM_CAP; break; }
    k++;
    c1 = c2;
    sigma = k * sigma;
    block_times_small(Vb, n, P, Js, Vn);
    memcpy(Vb, Vn, sizeof(double) * (size_t)n * P);
    csr_times_block(A, D, P, Y);
    st->spmm_count++;
    for (int64_t idx = 0; idx < (int64_t)n * P; ++idx) D[idx] = t * (Y[idx] - xi * D[idx]) / (double)s_int + Vb[idx];
    c2 = norm_inf(D, n, P) / sigma;
    for (int64_t idx = 0; idx < (int64_t)n * P; ++idx) S[idx] = S[idx] + D[idx] / sigma;
  }
  st->series_terms = k;
  double* F = (double*)malloc(sizeof(double) * (size_t)n * 2);
  double* E = (double*)malloc(sizeof(double) * (size_t)n * 2);
  double* Yf = (double*)malloc(sizeof(double) * (size_t)n * 2);
  memcpy(F, S, sizeof(double) * (size_t)n);
  memcpy(F + n, S + (int64_t)p * n, sizeof(double) * (size_t)n);
  if (status == ORC_OK) {
    csr_times_block(A, F, 1, Yf);
    st->spmm_count++;
    for (int64_t q = 0; q < n; ++q) F[q] = t * Yf[q] + Vin[q];
  }
  double* Sn = (double*)malloc(sizeof(double) * (size_t)n * P);
  for (int j = 1; j <= s_int - 1 && status == ORC_OK; ++j) {
    memcpy(E, F, sizeof(double) * (size_t)n * 2);
    int kk = 0;
    double d1 = INFINITY, d2 = norm_inf(F, n, 2);
    for (;;) {
      const double nE = norm_inf(E, n, 2);
      if (!isfinite(d2) || !isfinite(nE)) { status = ORC_NONFINITE; break; }
      if (!(d1 + d2 > tol * nE)) break;
      if (kk >= max_terms) { status = ORC_TERM_CAP; break; }
      kk++;
      d1 = d2;
      csr_times_block(A, F, 2, Yf);
      st->spmm_count++;
      for (int64_t idx = 0; idx < n * 2; ++idx) F[idx] = t * (Yf[idx] - xi * F[idx]) / ((double)s_int * kk);
      d2 = norm_inf(F, n, 2);
      for (int64_t idx = 0; idx < n * 2; ++idx) E[idx] = E[idx] + F[idx];
    }
    st->recovery_terms += kk;
    if (kk > st->max_inner_terms) st->max_inner_terms = kk;
    if (status != ORC_OK) break;
    for (int64_t idx = 0; idx < n * 2; ++idx) E[idx] = mu * E[idx];
    block_times_small(S, n, P, Jt, Sn);
    memcpy(S, Sn, sizeof(double) * (size_t)n * P);
    for (int64_t q = 0; q < n; ++q) {
      F[q] = E[q];
      F[n + q] = E[n + q] + S[(int64_t)p * n + q];
    }
  }
  for (int64_t q = 0; q < n; ++q) w_out[q] = (p == 0) ? F[q] : F[q] + alpha * F[n + q];
  st->status = status;
  free(Vb); free(aJ); free(Jt); free(Pw); free(Tmp); free(Js); free(S); free(D); free(Y); free(Vn);
  free(F); free(E); free(Yf); free(Sn);
  return status;
}

#ifdef _OPENMP
#include <omp.h>
#endif
int orc_set_threads(int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
  return omp_get_max_threads();
#else
  (void)nthreads;
  return 1;
#endif
}
