// Algorithms 1 and 3 for operators given as functions (phic_fn_* in include/phicomb.h).
//
// The caller's function enqueues Y = A X; everything else is the library's.  Algorithm 3 runs as one CUDA
// graph per call:
//
//   fn_setup -> fn_series_init -> WHILE(series) { apply(D) ; fn_series_term }
//            -> apply(S blk 0) ; fn_first
//            -> WHILE(steps) { fn_step_init ; WHILE(terms) { apply(G) ; fn_recover_term } ; fn_refresh }
//            -> fn_output
//
// Each kernel is a plain grid-stride pass (one thread per row, the row's columns in a loop).  The last
// block to finish a pass (counted with an atomic) reads the pass's infinity norms, takes the method's
// decision exactly as the persistent kernels do (the truncation test of Section 3 after every term, the
// recovery's step count s - 1), prepares the next term's scalars and sets the WHILE node's condition with
// cudaGraphSetConditional, so no Taylor term returns to the host.  The arithmetic per element is that of
// the stored-operator path: the products enter as B X = (A X - xi X) 2^-eA, with eA from the caller's
// bound of ||A||_inf; the recovery carries G_k = B^k F_0 with coefficients c_k = (t 2^eA / s)^k / k! rounded
// without bias, and its undo factors are compensated (see solve_body.cuh).
//
// Algorithm 1 runs its products on the caller's stream and its guard and Brent's method on the host, one
// synchronisation per basis vector and per objective evaluation (Algorithm 1 runs once per operator; the
// paper reuses its output across calls).  Its device passes are those of the selection kernel: the same
// fixed chunks of rows for every sum of squares, and the same objective coefficients.
#include <cuda_runtime.h>

#include <cfloat>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "layout.h"
#include "phicomb.h"
#include "select_body.cuh"
#include "select_coef.cuh"
#include "solve_body.cuh"

namespace phic {
void count_launch();

namespace {

constexpr int kFnBlock = kBlock;

// Device state of one function-operator solve (zeroed before the graph runs).
struct FnState {
  int status, s_int, eA, k, j, series_terms, max_inner, go;
  long long rec_terms;
  unsigned count;                 // blocks done with the current pass (the last one decides)
  unsigned pad;
  unsigned long long slot[3];     // pass maxima of non-negative doubles as bits; slot 2: non-finite flag
  double xi, s_used;
  double c1, c2, nrm, cF;         // truncation test: c1, c2 and ||S|| (series) or ||E|| (recovery)
  double tc[PHIC_MAX_R], cA[PHIC_MAX_R], cD[PHIC_MAX_R], cV[PHIC_MAX_R];
  double kd[PHIC_MAX_R], ka[PHIC_MAX_R], kt[PHIC_MAX_R];  // the series' coefficients of the current term
  double tBh[PHIC_MAX_R], tBl[PHIC_MAX_R];                 // t_i 2^eA / s in double-double
  double ch[PHIC_MAX_R], cl[PHIC_MAX_R];                   // c_k in double-double
  double coef[PHIC_MAX_R];                                 // c_k rounded to the tile type (exact as a double)
  double pmh[PHIC_MAX_R], pml[PHIC_MAX_R];                 // applied undo factors: (pmh + pml) 2^pe
  int pe[PHIC_MAX_R];
};

template <typename T>
struct FnArgs {
  int n, p, r, w_s, w_f, ld_s, ld_f, no_v0, max_terms;
  double tol, norm_bound;
  double t[PHIC_MAX_R], alpha[PHIC_MAX_R];
  const phic_params* params;
  const T* Vin;
  T* W;
  T *V, *D, *S, *Y, *G, *E;
  FnState* st;
  phic_stats* stats;
  cudaGraphConditionalHandle h_series, h_steps, h_terms;
};

// Block maxima of a pass into st.slot[idx] (thread 0 of each block), then the last-block test: true in
// every thread of the block that finished last, after which every block's slot update is visible to it.
__device__ __forceinline__ void pass_max(FnState* st, int idx, double v) {
  unsigned long long u = block_max_u64(dbits(v));
  if (threadIdx.x == 0 && u) atomicMax(&st->slot[idx], u);
}
__device__ __forceinline__ bool last_block(FnState* st) {
  __shared__ int s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(&st->count, 1u);
    s_last = prev == gridDim.x - 1;
    if (s_last) __threadfence();
  }
  __syncthreads();
  return s_last != 0;
}
__device__ __forceinline__ double slot_read(FnState* st, int idx) {
  return bitsd(*(volatile unsigned long long*)&st->slot[idx]);
}
__device__ __forceinline__ void pass_reset(FnState* st) {
  st->slot[0] = st->slot[1] = st->slot[2] = 0ull;
  st->count = 0u;
}

// ---- series ---------------------------------------------------------------------------------------
template <typename T>
__global__ void fn_setup(FnArgs<T> a) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  FnState& st = *a.st;
  // as the stored-operator path: xi in FP32 for FP32 tiles (N3), s raised for FP32 steps (R19)
  const double xi = sizeof(T) == 4 ? (double)__double2float_rn(a.params->xi) : a.params->xi;
  double s = a.params->s;
  if (sizeof(T) == 4) {
    const double nu = a.params->s0 * a.params->f_star;
    if (nu > 0.0 && isfinite(nu)) s = fmax(s, nu / kTheta32);
  }
  int bad = !isfinite(xi) || !(s >= 0.0) || !isfinite(s);
  double tmax = 0.0;
  for (int i = 0; i < a.r; ++i) tmax = fmax(tmax, fabs(a.t[i]));
  double sint = ceil(s * tmax);
  if (!(sint >= 1.0)) sint = 1.0;
  if (sint > 2147483647.0) bad = 1;
  const int si = bad ? 1 : (int)sint;
  for (int i = 0; i < a.r; ++i) {
    st.tc[i] = a.t[i] / si;
    st.cA[i] = a.alpha[i] / si;
    st.cD[i] = -(xi * a.t[i]) / si;
    st.cV[i] = exp(xi * a.t[i] / si) / si;
  }
  const double bound = a.norm_bound + fabs(xi);  // >= ||A - xi I||_inf
  st.eA = (bound > 0.0 && isfinite(bound)) ? ilogb(bound) + 1 : 0;
  st.xi = xi;
  st.s_used = s;
  st.s_int = si;
  st.status = bad ? PHIC_INVALID_ARG : PHIC_OK;
  st.k = 1;
  st.c1 = INFINITY;
}

// The series test after term k (c2 = ||D_k||, nrm = ||S||), preparing term k+1 (last block, thread 0).
template <typename T>
__device__ void series_decide(const FnArgs<T>& a, FnState& st) {
  int go = 0;
  if (st.status == PHIC_OK && (!isfinite(st.c2) || !isfinite(st.nrm))) st.status = PHIC_NONFINITE;
  if (st.status == PHIC_OK && st.c1 + st.c2 > a.tol * st.nrm) {
    if (st.k >= a.max_terms) {
      st.status = PHIC_TERM_CAP;
    } else {
      st.k += 1;
      st.c1 = st.c2;
      go = 1;
      const double sB = ldexp(1.0, st.eA);
      for (int i = 0; i < a.r; ++i) {
        st.kd[i] = (double)(T)(st.cD[i] / st.k);
        st.ka[i] = (double)(T)(st.cA[i] / st.k);
        st.kt[i] = (double)(T)(st.tc[i] * sB / st.k);
      }
    }
  }
  st.go = go;
  st.series_terms = st.k;
  cudaGraphSetConditional(a.h_series, go ? 1u : 0u);
}

// k = 1: V = D = S = the reordered, replicated and scaled inputs [v0, vp, ..., v1] (column (b, i) scaled by
// e^(xi t_i / s) / s).
template <typename T>
__global__ void __launch_bounds__(kFnBlock) fn_series_init(FnArgs<T> a) {
  FnState* st = a.st;
  double mx = 0.0;
  if (st->status == PHIC_OK) {
    for (long long row = (long long)blockIdx.x * blockDim.x + threadIdx.x; row < a.n;
         row += (long long)gridDim.x * blockDim.x) {
      double rs = 0.0;
      const size_t o = (size_t)row * a.ld_s;
      for (int c = 0; c < a.w_s; ++c) {
        const int b = c / a.r, i = c - b * a.r;
        const T* src = b == 0 ? (a.no_v0 ? nullptr : a.Vin) : a.Vin + (size_t)(a.p + 1 - b - a.no_v0) * a.n;
        const T x = src ? src[row] * (T)st->cV[i] : T(0);
        a.V[o + c] = x;
        a.D[o + c] = x;
        a.S[o + c] = x;
        rs += fabs((double)x);
      }
      mx = fmax(mx, rs);
    }
  }
  pass_max(st, 0, mx);
  if (last_block(st) && threadIdx.x == 0) {
    st->c2 = slot_read(st, 0);
    st->nrm = st->c2;
    pass_reset(st);
    series_decide(a, *st);
  }
}

// k >= 2, after Y = A D:  V <- V Jsh;  D <- B D (I kron T/s) 2^eA / k + V;  S <- S + D  (divided by k!).
template <typename T>
__global__ void __launch_bounds__(kFnBlock) fn_series_term(FnArgs<T> a) {
  FnState* st = a.st;
  const T xiT = (T)st->xi, sB = (T)ldexp(1.0, -st->eA);
  double mD = 0.0, mS = 0.0;
  for (long long row = (long long)blockIdx.x * blockDim.x + threadIdx.x; row < a.n;
       row += (long long)gridDim.x * blockDim.x) {
    const size_t o = (size_t)row * a.ld_s;
    double pD = 0.0, pS = 0.0;
    // from the last column down, so that block b-1 of V is still the old one when block b reads it
    for (int c = a.w_s - 1; c >= 0; --c) {
      const int b = c / a.r, i = c - b * a.r;
      const T acc = fma(-xiT, a.D[o + c], a.Y[o + c]) * sB;  // (B D)(row, c)
      T v = (T)st->kd[i] * a.V[o + c];
      if (b >= 2) v = fma((T)st->ka[i], a.V[o + c - a.r], v);
      const T d = fma(acc, (T)st->kt[i], v);
      const T sn = a.S[o + c] + d;
      a.V[o + c] = v;
      a.D[o + c] = d;
      a.S[o + c] = sn;
      pD += fabs((double)d);
      pS += fabs((double)sn);
    }
    mD = fmax(mD, pD);
    mS = fmax(mS, pS);
  }
  pass_max(st, 0, mD);
  pass_max(st, 1, mS);
  if (last_block(st) && threadIdx.x == 0) {
    st->c2 = slot_read(st, 0);
    st->nrm = slot_read(st, 1);
    pass_reset(st);
    series_decide(a, *st);
  }
}

// ---- recovery ---------------------------------------------------------------------------------------
// c_k of every combination, rounded without bias (the recursion and the rounding of next_coefs).
template <typename T>
__device__ void fn_coefs(FnState& st, int r, int k, int j) {
  for (int i = 0; i < r; ++i) {
    const DD tBd{st.tBh[i], st.tBl[i]};
    const DD cd = k == 1 ? tBd : dd_over_d(dd_times(DD{st.ch[i], st.cl[i]}, tBd), (double)k);
    st.ch[i] = cd.h;
    st.cl[i] = cd.l;
    const CoefEntry<T> e = coef_entry<T>(cd);
    const unsigned long long key = ((unsigned long long)j << 32) ^ ((unsigned long long)k << 8) ^ (unsigned long long)i;
    st.coef[i] = (double)((unsigned)(unit_bits(key) >> 32) < e.thr ? e.alt : e.base);
  }
}

// The recovery test after term k (c2 = ||F_k||, nrm = ||E||), preparing term k+1.
template <typename T>
__device__ void recover_decide(const FnArgs<T>& a, FnState& st) {
  int go = 0;
  if (st.status == PHIC_OK && (!isfinite(st.c2) || !isfinite(st.nrm))) st.status = PHIC_NONFINITE;
  if (st.status == PHIC_OK && st.c1 + st.c2 > a.tol * st.nrm) {
    if (st.k >= a.max_terms) {
      st.status = PHIC_TERM_CAP;
    } else {
      st.k += 1;
      st.c1 = st.c2;
      go = 1;
      fn_coefs<T>(st, a.r, st.k, st.j);
    }
  }
  if (!go) {
    st.rec_terms += st.k;
    st.max_inner = st.k > st.max_inner ? st.k : st.max_inner;
  }
  cudaGraphSetConditional(a.h_terms, go ? 1u : 0u);
}

__device__ __forceinline__ int col_comb(int c, int r) { return c < r ? c : c - r; }

// After Y = A S(:, blk 0):  F = [A S(:, blk 0) T + v0 1^T, S(:, blk p)] (unshifted A, t undivided).
template <typename T>
__global__ void __launch_bounds__(kFnBlock) fn_first(FnArgs<T> a) {
  FnState* st = a.st;
  double mx = 0.0;
  for (long long row = (long long)blockIdx.x * blockDim.x + threadIdx.x; row < a.n;
       row += (long long)gridDim.x * blockDim.x) {
    const size_t os = (size_t)row * a.ld_s, of = (size_t)row * a.ld_f;
    const T v0 = a.no_v0 ? T(0) : a.Vin[row];
    double rs = 0.0;
    for (int c = 0; c < a.w_f; ++c) {
      const int i = col_comb(c, a.r);
      const T v = c < a.r ? fma(a.Y[os + i], (T)a.t[i], v0) : a.S[os + a.p * a.r + i];
      a.G[of + c] = v;
      rs += fabs((double)v);
    }
    mx = fmax(mx, rs);
  }
  pass_max(st, 0, mx);
  if (last_block(st) && threadIdx.x == 0) {
    FnState& s = *st;
    s.cF = slot_read(st, 0);
    pass_reset(st);
    const double sB = ldexp(1.0, s.eA);
    for (int i = 0; i < a.r; ++i) {
      const DD tBd = dd_over_d(DD{a.t[i] * sB, 0.0}, (double)s.s_int);
      s.tBh[i] = tBd.h;
      s.tBl[i] = tBd.l;
      s.pmh[i] = 1.0;
      s.pml[i] = 0.0;
      s.pe[i] = 0;
    }
    s.j = 0;
    const int go = s.status == PHIC_OK && s.s_int > 1;
    cudaGraphSetConditional(a.h_steps, go ? 1u : 0u);
  }
}

// Start of recovery step j: E = F, k = 0, c1 = inf; the first term always runs.
template <typename T>
__global__ void fn_step_init(FnArgs<T> a) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  FnState& st = *a.st;
  st.j += 1;
  st.k = 0;
  st.c1 = INFINITY;
  st.c2 = st.cF;
  st.nrm = st.cF;
  int go = 0;
  if (st.status == PHIC_OK && st.j <= st.s_int - 1) {
    if (!isfinite(st.cF)) {
      st.status = PHIC_NONFINITE;
    } else {
      st.k = 1;
      st.c1 = st.c2;
      go = 1;
      fn_coefs<T>(st, a.r, 1, st.j);
    }
  }
  cudaGraphSetConditional(a.h_terms, go ? 1u : 0u);
}

// After Y = A G_(k-1):  G_k = B G_(k-1);  E <- E + c_k G_k  (E = F on the first term).
template <typename T>
__global__ void __launch_bounds__(kFnBlock) fn_recover_term(FnArgs<T> a) {
  FnState* st = a.st;
  const T xiT = (T)st->xi, sB = (T)ldexp(1.0, -st->eA);
  const int k = st->k;
  __shared__ T s_coef[PHIC_MAX_R];
  if (threadIdx.x < (unsigned)a.r) s_coef[threadIdx.x] = (T)st->coef[threadIdx.x];
  __syncthreads();
  double mF = 0.0, mE = 0.0;
  for (long long row = (long long)blockIdx.x * blockDim.x + threadIdx.x; row < a.n;
       row += (long long)gridDim.x * blockDim.x) {
    const size_t o = (size_t)row * a.ld_f;
    double pF = 0.0, pE = 0.0;
    for (int c = 0; c < a.w_f; ++c) {
      const T cc = s_coef[col_comb(c, a.r)];
      const T g0 = a.G[o + c];
      const T g = fma(-xiT, g0, a.Y[o + c]) * sB;
      const T e = fma(cc, g, k == 1 ? g0 : a.E[o + c]);
      a.G[o + c] = g;
      a.E[o + c] = e;
      pF += fabs((double)cc) * fabs((double)g);
      pE += fabs((double)e);
    }
    mF = fmax(mF, pF);
    mE = fmax(mE, pE);
  }
  pass_max(st, 0, mF);
  pass_max(st, 1, mE);
  if (last_block(st) && threadIdx.x == 0) {
    st->c2 = slot_read(st, 0);
    st->nrm = slot_read(st, 1);
    pass_reset(st);
    recover_decide(a, *st);
  }
}

// End of recovery step j:  F = E mu_j + S Jt^j e_p  (mu_j compensated), then whether another step runs.
template <typename T>
__global__ void __launch_bounds__(kFnBlock) fn_refresh(FnArgs<T> a) {
  FnState* st = a.st;
  const int j = st->j, r = a.r, p = a.p;
  __shared__ T s_mu[PHIC_MAX_R];
  __shared__ T s_cj[PHIC_MAX_P + 1][PHIC_MAX_R];
  __shared__ double s_pm[PHIC_MAX_R][2];
  __shared__ int s_pe[PHIC_MAX_R];
  if (threadIdx.x < (unsigned)r) {  // every block forms the same factors; the last block keeps the product
    const int i = threadIdx.x;
    const DD x = dd_over_d(dd_prod(st->xi, a.t[i]), (double)st->s_int);
    const DD y = dd_times(dd_times_d(x, (double)j), DD{kLog2eHi, kLog2eLo});
    const double N = rint(y.h);
    T mu = (T)exp(x.h);
    double ph = st->pmh[i], pl = st->pml[i];
    int pe = st->pe[i];
    if (fabs(N) < 1e6) {
      const double f = (y.h - N) + y.l;
      double q = exp2(f) / ph;
      q -= q * (pl / ph);
      const double m = ldexp(q, (int)N - pe);
      const T muT = (T)m;
      const DD np = dd_times_d(DD{ph, pl}, (double)muT);
      if (muT != T(0) && isfinite(m) && np.h != 0.0 && isfinite(np.h)) {
        int ex = 0;
        ph = frexp(np.h, &ex);
        pl = ldexp(np.l, -ex);
        pe += ex;
        mu = muT;
      }
    }
    s_mu[i] = mu;
    s_pm[i][0] = ph;
    s_pm[i][1] = pl;
    s_pe[i] = pe;
  }
  for (int idx = threadIdx.x; idx < p * r; idx += blockDim.x) {  // block p of S Jt^j (J nilpotent)
    const int aa = 1 + idx / r, i = idx % r;
    const double x = (double)j * a.alpha[i] / st->s_int;
    double c = 1.0;
    for (int q = 1; q <= p - aa; ++q) c = c * x / q;
    s_cj[aa][i] = (T)c;
  }
  __syncthreads();
  double mx = 0.0;
  for (long long row = (long long)blockIdx.x * blockDim.x + threadIdx.x; row < a.n;
       row += (long long)gridDim.x * blockDim.x) {
    const size_t of = (size_t)row * a.ld_f, os = (size_t)row * a.ld_s;
    double rs = 0.0;
    for (int c = 0; c < a.w_f; ++c) {
      const int i = col_comb(c, r);
      T v = a.E[of + c] * s_mu[i];
      if (c >= r)
        for (int aa = 1; aa <= p; ++aa) v = fma(a.S[os + aa * r + i], s_cj[aa][i], v);
      a.G[of + c] = v;
      rs += fabs((double)v);
    }
    mx = fmax(mx, rs);
  }
  pass_max(st, 0, mx);
  if (last_block(st) && threadIdx.x == 0) {
    FnState& s = *st;
    s.cF = slot_read(st, 0);
    pass_reset(st);
    for (int i = 0; i < r; ++i) {
      s.pmh[i] = s_pm[i][0];
      s.pml[i] = s_pm[i][1];
      s.pe[i] = s_pe[i];
    }
    const int go = s.status == PHIC_OK && j < s.s_int - 1;
    cudaGraphSetConditional(a.h_steps, go ? 1u : 0u);
  }
}

// w_i = F(:, i) + alpha_i F(:, r+i)  (p = 0: w_i = F(:, i)); the record.
template <typename T>
__global__ void __launch_bounds__(kFnBlock) fn_output(FnArgs<T> a) {
  const FnState* st = a.st;
  if (st->status == PHIC_OK) {
    const long long total = (long long)a.n * a.r;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
      const int i = (int)(idx / a.n), row = (int)(idx - (long long)i * a.n);
      const T* f = a.G + (size_t)row * a.ld_f;
      a.W[idx] = a.p == 0 ? f[i] : fma((T)a.alpha[i], f[a.r + i], f[i]);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && a.stats) {
    phic_stats& s = *a.stats;
    s.status = st->status;
    s.s_int = st->s_int;
    s.series_terms = st->series_terms;
    s.max_inner_terms = st->max_inner;
    s.recovery_terms = st->rec_terms;
    s.spmm_count = (long long)(st->series_terms - 1) + 1 + st->rec_terms;
    s.xi = st->xi;
    s.s = st->s_used;
    s.op_format = PHIC_OP_FUNCTION;
    s.op_slots = 0;
  }
}

// ---- the graph --------------------------------------------------------------------------------------
struct FnLayout {
  size_t state, V, D, S, Y, G, E, total;
  int ld_s, ld_f;
};
inline FnLayout fn_layout(int64_t n, int p, int r, int prec) {
  FnLayout L;
  const size_t es = prec == PHIC_F32 ? 4 : 8;
  const int w_s = (p + 1) * r, w_f = p > 0 ? 2 * r : r;
  L.ld_s = (w_s + 1) & ~1;  // even strides: rows start on 16-byte boundaries for the caller's loads
  L.ld_f = (w_f + 1) & ~1;
  const size_t tS = align_up((size_t)n * L.ld_s * es), tF = align_up((size_t)n * L.ld_f * es);
  size_t off = 0;
  L.state = off; off += align_up(sizeof(FnState));
  L.V = off; off += tS;
  L.D = off; off += tS;
  L.S = off; off += tS;
  L.Y = off; off += tS;
  L.G = off; off += tF;
  L.E = off; off += tF;
  L.total = off;
  return L;
}

// A WHILE node at the current point of the capture on stream cs, its body filled by body(bs) captured on bs.
template <typename Body>
cudaError_t add_while(cudaStream_t cs, cudaStream_t bs, cudaGraphConditionalHandle h, Body&& body) {
  cudaStreamCaptureStatus status;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(cs, &status, nullptr, &g, &deps, nullptr, &ndeps);
  if (e != cudaSuccess) return e;
  if (status != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
  cudaGraphNodeParams prm{};
  prm.type = cudaGraphNodeTypeConditional;
  prm.conditional.handle = h;
  prm.conditional.type = cudaGraphCondTypeWhile;
  prm.conditional.size = 1;
  cudaGraphNode_t node;
  e = cudaGraphAddNode(&node, g, deps, nullptr, ndeps, &prm);
  if (e != cudaSuccess) return e;
  e = cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
  if (e != cudaSuccess) return e;
  cudaGraph_t bodyg = prm.conditional.phGraph_out[0];
  e = cudaStreamBeginCaptureToGraph(bs, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t eb = body(bs);
  cudaGraph_t out = nullptr;
  e = cudaStreamEndCapture(bs, &out);
  return eb != cudaSuccess ? eb : e;
}

template <typename T>
cudaError_t fn_graph_solve(const phic_fn_op* A, FnArgs<T> a, cudaStream_t user_stream) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  long long need = ((long long)a.n + kFnBlock - 1) / kFnBlock;
  const int grid = (int)(need < (long long)sms * 8 ? (need < 1 ? 1 : need) : (long long)sms * 8);
  cudaGraph_t g = nullptr;
  cudaGraphExec_t x = nullptr;
  cudaStream_t cs = nullptr, bs = nullptr, bs2 = nullptr;
  const int prec = sizeof(T) == 4 ? PHIC_F32 : PHIC_F64;
  auto apply = [&](const T* X, int ldx, int w, cudaStream_t s) -> cudaError_t {
    return A->apply(A->ctx, X, ldx, a.Y, ldx, w, prec, reinterpret_cast<phic_stream_t>(s)) == 0 ? cudaSuccess
                                                                                               : cudaErrorLaunchFailure;
  };
  auto k_launch = [&](auto kernel, int blocks, cudaStream_t s) -> cudaError_t {
    kernel<<<blocks, kFnBlock, 0, s>>>(a);
    count_launch();
    return cudaGetLastError();
  };
  do {
    if ((e = cudaGraphCreate(&g, 0)) != cudaSuccess) break;
    if ((e = cudaGraphConditionalHandleCreate(&a.h_series, g, 1, cudaGraphCondAssignDefault)) != cudaSuccess) break;
    if ((e = cudaGraphConditionalHandleCreate(&a.h_steps, g, 0, cudaGraphCondAssignDefault)) != cudaSuccess) break;
    if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess) break;
    if ((e = cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking)) != cudaSuccess) break;
    if ((e = cudaStreamCreateWithFlags(&bs2, cudaStreamNonBlocking)) != cudaSuccess) break;
    if ((e = cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
      break;
    cudaError_t ec = cudaSuccess;
    do {
      if ((ec = cudaMemsetAsync(a.st, 0, sizeof(FnState), cs)) != cudaSuccess) break;
      if ((ec = k_launch(fn_setup<T>, 1, cs)) != cudaSuccess) break;
      if ((ec = k_launch(fn_series_init<T>, grid, cs)) != cudaSuccess) break;
      ec = add_while(cs, bs, a.h_series, [&](cudaStream_t s) {
        cudaError_t eb = apply(a.D, a.ld_s, a.w_s, s);
        return eb != cudaSuccess ? eb : k_launch(fn_series_term<T>, grid, s);
      });
      if (ec != cudaSuccess) break;
      if ((ec = apply(a.S, a.ld_s, a.r, cs)) != cudaSuccess) break;  // A S(:, blk 0): the first r columns
      if ((ec = k_launch(fn_first<T>, grid, cs)) != cudaSuccess) break;
      ec = add_while(cs, bs, a.h_steps, [&](cudaStream_t s) {
        cudaError_t eb = cudaSuccess;
        cudaStreamCaptureStatus cst;
        cudaGraph_t bg = nullptr;
        if ((eb = cudaStreamGetCaptureInfo(s, &cst, nullptr, &bg, nullptr, nullptr, nullptr)) != cudaSuccess) return eb;
        if ((eb = cudaGraphConditionalHandleCreate(&a.h_terms, bg, 0, cudaGraphCondAssignDefault)) != cudaSuccess)
          return eb;
        if ((eb = k_launch(fn_step_init<T>, 1, s)) != cudaSuccess) return eb;
        eb = add_while(s, bs2, a.h_terms, [&](cudaStream_t s2) {
          cudaError_t ei = apply(a.G, a.ld_f, a.w_f, s2);
          return ei != cudaSuccess ? ei : k_launch(fn_recover_term<T>, grid, s2);
        });
        if (eb != cudaSuccess) return eb;
        return k_launch(fn_refresh<T>, grid, s);
      });
      if (ec != cudaSuccess) break;
      ec = k_launch(fn_output<T>, grid, cs);
    } while (false);
    cudaGraph_t out = nullptr;
    e = cudaStreamEndCapture(cs, &out);
    if (ec != cudaSuccess) e = ec;
    if (e != cudaSuccess) break;
    if ((e = cudaGraphInstantiate(&x, g, 0)) != cudaSuccess) break;
    e = cudaGraphLaunch(x, user_stream);
  } while (false);
  if (x) cudaGraphExecDestroy(x);  // released once the launch completes
  if (g) cudaGraphDestroy(g);
  if (cs) cudaStreamDestroy(cs);
  if (bs) cudaStreamDestroy(bs);
  if (bs2) cudaStreamDestroy(bs2);
  return e;
}

// ---- Algorithm 1 ------------------------------------------------------------------------------------
// Sum of squares of y = f(row) per fixed chunk of kChunk rows into part[chunk] (as chunk_pass).
template <typename F>
__device__ __forceinline__ void fn_chunks(int n, Ssq* part, F&& f) {
  const int nch = chunk_count(n);
  for (int c = blockIdx.x; c < nch; c += gridDim.x) {
    Ssq acc = ssq_empty();
#pragma unroll
    for (int u = 0; u < kChunk / kBlock; ++u) {
      const long long row = (long long)c * kChunk + u * kBlock + threadIdx.x;
      if (row < n) ssq_add(acc, f(row));
    }
    const Ssq blk = block_ssq(acc);
    if (threadIdx.x == 0) part[c] = blk;
  }
}

// V_0 = v (given, or components 2u - 1 with u from splitmix64(seed, i)); its sum of squares.
__global__ void __launch_bounds__(kBlock) fnsel_init(int n, const double* v, uint64_t seed, double* Vb, Ssq* part) {
  fn_chunks(n, part, [&](long long row) {
    const double x = v ? v[row] : 2.0 * ((double)(splitmix64_at(seed, (uint64_t)row) >> 11) * 0x1.0p-53) - 1.0;
    Vb[vidx(0, n, row)] = x;
    return x;
  });
}
// V_k <- V_k * factor, or V_k / factor with divide (factor 1: unchanged), and its sum of squares.
__global__ void __launch_bounds__(kBlock) fnsel_scale(int n, int k, double factor, int divide, double* Vb, Ssq* part) {
  fn_chunks(n, part, [&](long long row) {
    double x = Vb[vidx(k, n, row)];
    if (factor != 1.0) {
      x = divide ? x / factor : x * factor;
      Vb[vidx(k, n, row)] = x;
    }
    return x;
  });
}
// V_j <- V_j s0^-j for j = 1..r (the factors as the selection kernel forms them).
__global__ void __launch_bounds__(kBlock) fnsel_normalise(int n, int r, double s0, double* Vb) {
  __shared__ double f[kMaxM + 1];
  if (threadIdx.x >= 1 && threadIdx.x <= r) f[threadIdx.x] = exp(-(double)threadIdx.x * log(s0));
  __syncthreads();
  for (long long row = (long long)blockIdx.x * blockDim.x + threadIdx.x; row < n; row += (long long)gridDim.x * blockDim.x)
    for (int j = 1; j <= r; ++j) Vb[vidx(j, n, row)] *= f[j];
}
// One objective pass: y = sum_k binom(m,k) z^(m-k) V_k per row, its sum of squares.
__global__ void __launch_bounds__(kBlock) fnsel_objective(int n, int m, double z, const double* Vb, Ssq* part) {
  __shared__ double binom[kMaxM + 1];
  __shared__ double coef[kMaxM + 1];
  if (threadIdx.x == 0) binomial_row(m, binom);
  __syncthreads();
  if (threadIdx.x <= (unsigned)m) coef[threadIdx.x] = objective_coef(binom[threadIdx.x], z, m - (int)threadIdx.x);
  __syncthreads();
  const double2* __restrict__ Vp2 = reinterpret_cast<const double2*>(Vb);
  const int pairs = (m + 1) >> 1;
  fn_chunks(n, part, [&](long long row) {
    double y = 0.0;
    for (int jj = 0; jj < pairs; ++jj) {
      const double2 v = Vp2[(size_t)jj * n + row];
      y = fma(coef[2 * jj], v.x, y);
      y = fma(coef[2 * jj + 1], v.y, y);
    }
    if ((m + 1) & 1) y = fma(coef[m], Vb[vidx(m, n, row)], y);
    return y;
  });
}
// log of the 2-norm from the chunks' partials in their fixed order (one block).
__global__ void __launch_bounds__(kBlock) fnsel_combine(int n, const Ssq* part, double* out) {
  const Ssq tot = gather_chunks(part, 0, n);
  if (threadIdx.x == 0) *out = ssq_log_norm(tot);
}

struct FnSelLayout {
  size_t basis, part, result, total;
};
inline int host_chunks(int64_t n) { return (int)((n + kChunk - 1) / kChunk); }
inline size_t host_vidx(int k, int64_t n) { return ((size_t)(k >> 1) * (size_t)n) * 2 + (size_t)(k & 1); }
inline FnSelLayout fnsel_layout(int64_t n, int m) {
  FnSelLayout L;
  size_t off = 0;
  L.basis = off; off += align_up((size_t)n * (m + 1 + ((m + 1) & 1)) * sizeof(double));
  L.part = off; off += align_up((size_t)host_chunks(n) * sizeof(Ssq));
  L.result = off; off += align_up(sizeof(double));
  L.total = off;
  return L;
}

}  // namespace
}  // namespace phic

using namespace phic;

extern "C" {

phic_status phic_fn_select_workspace_size(int64_t n, int32_t m, size_t* bytes) {
  if (!bytes || n < 1 || n >= (int64_t)INT32_MAX || m < 1 || m > 128) return PHIC_INVALID_ARG;
  *bytes = fnsel_layout(n, m).total;
  return PHIC_OK;
}

phic_status phic_fn_select_params(const phic_fn_op* A, const phic_select_opts* opts, const double* v, void* ws,
                                  size_t ws_bytes, phic_params* params_dev, phic_stream_t stream) {
  phic_select_opts o;
  if (opts) o = *opts; else phic_select_opts_default(&o);
  if (!A || !A->apply || A->n < 1 || A->n >= (int64_t)INT32_MAX || !params_dev || !ws || !aligned(ws) ||
      !select_opts_ok(o))
    return PHIC_INVALID_ARG;
  const int n = (int)A->n, m = o.m;
  const FnSelLayout L = fnsel_layout(n, m);
  if (ws_bytes < L.total) return PHIC_WORKSPACE_TOO_SMALL;
  char* base = static_cast<char*>(ws);
  double* Vb = reinterpret_cast<double*>(base + L.basis);
  Ssq* part = reinterpret_cast<Ssq*>(base + L.part);
  double* res = reinterpret_cast<double*>(base + L.result);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return PHIC_CUDA_ERROR;
  const int nch = host_chunks(n);
  const int grid = nch < sms * 4 ? nch : sms * 4;
  const int rgrid = (int)(((long long)n + kBlock - 1) / kBlock < sms * 8 ? ((long long)n + kBlock - 1) / kBlock : sms * 8);
  // log 2-norm of the last pass, read on the host
  auto lognorm = [&](double* out) -> bool {
    fnsel_combine<<<1, kBlock, 0, st>>>(n, part, res);
    count_launch();
    return cudaMemcpyAsync(out, res, sizeof(double), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
           cudaStreamSynchronize(st) == cudaSuccess;
  };
  auto product = [&](int k) -> bool {  // V_k = A V_(k-1), both pair-interleaved (row stride 2)
    return A->apply(A->ctx, Vb + host_vidx(k - 1, n), 2, Vb + host_vidx(k, n), 2, 1, PHIC_F64, stream) == 0;
  };
  phic_params out;
  std::memset(&out, 0, sizeof(out));
  out.status = PHIC_OK;
  auto finish = [&]() -> phic_status {
    return cudaMemcpyAsync(params_dev, &out, sizeof(out), cudaMemcpyHostToDevice, st) == cudaSuccess &&
                   cudaStreamSynchronize(st) == cudaSuccess
               ? PHIC_OK
               : PHIC_CUDA_ERROR;
  };
  // v and its normalisation: V_0 = v / ||v||, L_0
  double lg = 0.0;
  fnsel_init<<<grid, kBlock, 0, st>>>(n, v, o.seed, Vb, part);
  count_launch();
  if (!lognorm(&lg)) return PHIC_CUDA_ERROR;
  if (!std::isfinite(lg)) {
    out.status = PHIC_INVALID_ARG;
    return finish() == PHIC_OK ? PHIC_OK : PHIC_CUDA_ERROR;
  }
  std::vector<double> Lk(m + 1, 0.0);
  fnsel_scale<<<grid, kBlock, 0, st>>>(n, 0, std::exp(lg), 1, Vb, part);
  count_launch();
  if (!lognorm(&Lk[0])) return PHIC_CUDA_ERROR;
  // the guarded power basis: stop at the first k whose log-norm breaks the overflow/underflow guard
  double lmax = -INFINITY;
  for (int j = m / 2; j <= (m + 1) / 2; ++j)
    lmax = std::fmax(lmax, std::lgamma(m + 1.0) - std::lgamma(j + 1.0) - std::lgamma(m - j + 1.0));
  const double gmax = o.delta * std::log(DBL_MAX), gmin = o.delta * std::log(DBL_MIN);
  int r = 0;
  for (int k = 1; k <= m; ++k) {
    if (!product(k)) return PHIC_CUDA_ERROR;
    fnsel_scale<<<grid, kBlock, 0, st>>>(n, k, 1.0, 0, Vb, part);
    count_launch();
    double L = 0.0;
    if (!lognorm(&L)) return PHIC_CUDA_ERROR;
    if (L + 0.5 * std::log(k + 1.0) + lmax > gmax || L < gmin || std::isnan(L)) break;
    Lk[k] = L;
    r = k;
  }
  if (r == 0) {  // nothing accepted: xi = 0, s = 1
    out.xi = 0.0;
    out.s = 1.0;
    return finish();
  }
  // s0 from the last growth factors; V_j <- s0^-j V_j; the extension V_k = A V_(k-1) / s0
  int jr = r - 5 > 2 ? r - 5 : 2;
  if (r - jr <= 0) jr = r - 1 > 0 ? r - 1 : 0;
  const double s0 = std::exp((Lk[r] - Lk[jr]) / (double)(r - jr));
  fnsel_normalise<<<rgrid, kBlock, 0, st>>>(n, r, s0, Vb);
  count_launch();
  const double inv_s0 = 1.0 / s0;
  for (int k = r + 1; k <= m; ++k) {
    if (!product(k)) return PHIC_CUDA_ERROR;
    fnsel_scale<<<grid, kBlock, 0, st>>>(n, k, inv_s0, 0, Vb, part);
    count_launch();
  }
  if (cudaGetLastError() != cudaSuccess) return PHIC_CUDA_ERROR;
  // Brent's method on f(xi) over [-sqrt(n) s0, sqrt(n) s0]
  BrentSM br;
  const double half = std::sqrt((double)n) * s0;
  brent_start(br, -half, half, 1e-8 * s0, o.max_evals);
  while (true) {
    fnsel_objective<<<grid, kBlock, 0, st>>>(n, m, -br.u / s0, Vb, part);
    count_launch();
    double lf = 0.0;
    if (!lognorm(&lf)) return PHIC_CUDA_ERROR;
    brent_feed(br, lf == -INFINITY ? 0.0 : std::exp(lf / (double)m));
    if (br.done) break;
  }
  const double ltm = (std::log(o.tol) + std::lgamma(m + 1.0)) / (double)m;  // log (tol m!)^(1/m)
  out.xi = br.x;
  out.s = s0 * br.fx / std::exp(ltm);
  out.s0 = s0;
  out.f_star = br.fx;
  out.r = r;
  out.evals = br.evals;
  out.status = (std::isfinite(out.s) && std::isfinite(out.xi)) ? PHIC_OK : PHIC_NONFINITE;
  return finish();
}

phic_status phic_fn_solve_workspace_size(int64_t n, int32_t p, int32_t r, int32_t prec, size_t* bytes) {
  if (!bytes || n < 1 || n >= (int64_t)INT32_MAX || p < 0 || p > PHIC_MAX_P || r < 1 || r > PHIC_MAX_R ||
      (p + 1) * r > PHIC_MAX_WIDTH || (prec != PHIC_F64 && prec != PHIC_F32))
    return PHIC_INVALID_ARG;
  *bytes = fn_layout(n, p, r, prec).total;
  return PHIC_OK;
}

phic_status phic_fn_solve(const phic_fn_op* A, int32_t p, int32_t r, const void* V, const double* t,
                          const double* alpha, double tol, const phic_params* params_dev, uint32_t flags,
                          int32_t max_terms, void* W, void* ws, size_t ws_bytes, phic_stats* stats_dev,
                          int32_t prec, phic_stream_t stream) {
  if (!A || !A->apply || A->n < 1 || A->n >= (int64_t)INT32_MAX || A->prec != prec || !(A->norm_bound > 0.0) ||
      !std::isfinite(A->norm_bound) || p < 0 || p > PHIC_MAX_P || r < 1 || r > PHIC_MAX_R ||
      (p + 1) * r > PHIC_MAX_WIDTH || (prec != PHIC_F64 && prec != PHIC_F32) || !V || !t || !alpha || !W ||
      !params_dev || !ws || !aligned(ws) || !(tol > 0.0) || !std::isfinite(tol) || (flags & ~PHIC_NO_V0) ||
      ((flags & PHIC_NO_V0) && p == 0))
    return PHIC_INVALID_ARG;
  for (int i = 0; i < r; ++i)
    if (!std::isfinite(t[i]) || !std::isfinite(alpha[i])) return PHIC_INVALID_ARG;
  const FnLayout L = fn_layout(A->n, p, r, prec);
  if (ws_bytes < L.total) return PHIC_WORKSPACE_TOO_SMALL;
  char* base = static_cast<char*>(ws);
  auto fill = [&](auto& a) {
    using TT = std::remove_pointer_t<decltype(a.V)>;
    a.n = (int)A->n;
    a.p = p;
    a.r = r;
    a.w_s = (p + 1) * r;
    a.w_f = p > 0 ? 2 * r : r;
    a.ld_s = L.ld_s;
    a.ld_f = L.ld_f;
    a.no_v0 = (flags & PHIC_NO_V0) ? 1 : 0;
    a.max_terms = max_terms > 0 ? max_terms : 610;
    a.tol = tol;
    a.norm_bound = A->norm_bound;
    for (int i = 0; i < PHIC_MAX_R; ++i) {
      a.t[i] = i < r ? t[i] : 0.0;
      a.alpha[i] = i < r ? alpha[i] : 0.0;
    }
    a.params = params_dev;
    a.Vin = static_cast<const TT*>(V);
    a.W = static_cast<TT*>(W);
    a.V = reinterpret_cast<TT*>(base + L.V);
    a.D = reinterpret_cast<TT*>(base + L.D);
    a.S = reinterpret_cast<TT*>(base + L.S);
    a.Y = reinterpret_cast<TT*>(base + L.Y);
    a.G = reinterpret_cast<TT*>(base + L.G);
    a.E = reinterpret_cast<TT*>(base + L.E);
    a.st = reinterpret_cast<FnState*>(base + L.state);
    a.stats = stats_dev;
  };
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (prec == PHIC_F64) {
    FnArgs<double> a{};
    fill(a);
    e = fn_graph_solve<double>(A, a, st);
  } else {
    FnArgs<float> a{};
    fill(a);
    e = fn_graph_solve<float>(A, a, st);
  }
  return e == cudaSuccess ? PHIC_OK : PHIC_CUDA_ERROR;
}

}  // extern "C"

// ---- phic_csr_apply ---------------------------------------------------------------------------------
namespace phic {
namespace {
template <typename TX, typename TV>
__global__ void __launch_bounds__(kBlock) csr_apply_kernel(int n, const int* __restrict__ rowptr,
                                                           const int* __restrict__ colidx, const TV* __restrict__ vals,
                                                           const TX* __restrict__ X, long long ldx, TX* __restrict__ Y,
                                                           long long ldy, int w) {
  const long long total = (long long)n * w;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int row = (int)(idx / w), c = (int)(idx - (long long)row * w);
    const int b0 = __ldg(rowptr + row), b1 = __ldg(rowptr + row + 1);
    TX acc = TX(0);
    for (int q = b0; q < b1; ++q) {
      const int col = __ldg(colidx + q);
      if ((unsigned)col < (unsigned)n) acc = fma((TX)__ldg(vals + q), X[(size_t)col * ldx + c], acc);
    }
    Y[(size_t)row * ldy + c] = acc;
  }
}
}  // namespace
}  // namespace phic

extern "C" int32_t phic_csr_apply(void* ctx, const void* X, int64_t ldx, void* Y, int64_t ldy, int32_t w,
                                  int32_t prec, phic_stream_t stream) {
  const phic_csr* A = static_cast<const phic_csr*>(ctx);
  if (!A || !X || !Y || w < 1 || ldx < w || ldy < w || A->n < 1) return 1;
  if (prec == PHIC_F32 && A->prec != PHIC_F32) return 1;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 1;
  const long long total = A->n * (long long)w;
  const long long need = (total + kBlock - 1) / kBlock;
  const int grid = (int)(need < (long long)sms * 8 ? need : (long long)sms * 8);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int n = (int)A->n;
  if (prec == PHIC_F64) {
    if (A->prec == PHIC_F64)
      csr_apply_kernel<double, double><<<grid, kBlock, 0, st>>>(n, A->rowptr, A->colidx, static_cast<const double*>(A->values),
                                                                static_cast<const double*>(X), ldx, static_cast<double*>(Y), ldy, w);
    else
      csr_apply_kernel<double, float><<<grid, kBlock, 0, st>>>(n, A->rowptr, A->colidx, static_cast<const float*>(A->values),
                                                               static_cast<const double*>(X), ldx, static_cast<double*>(Y), ldy, w);
  } else {
    csr_apply_kernel<float, float><<<grid, kBlock, 0, st>>>(n, A->rowptr, A->colidx, static_cast<const float*>(A->values),
                                                            static_cast<const float*>(X), ldx, static_cast<float*>(Y), ldy, w);
  }
  count_launch();
  return cudaGetLastError() == cudaSuccess ? 0 : 1;
}
