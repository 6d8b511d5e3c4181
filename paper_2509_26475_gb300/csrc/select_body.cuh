#pragma once
// Algorithm 1 of the paper (Section 3): selection of the shift xi* and the scaling s.
//
// One team of CTAs (the whole grid of a single launch, or a share of a batched launch) runs every step
// in FP64 whatever the precision of A's values:
//   1. v (given, or splitmix64 components 2u-1) normalised to a unit 2-norm: V_0;
//   2. the guarded power basis W_k = A V_{k-1}, L_k = log ||W_k||_2, stopped at the first k with
//      L_k + log(k+1)/2 + l_max > g_max or L_k < g_min (r = last accepted k);
//   3. s0 = exp((L_r - L_{j_r}) / (r - j_r)), j_r = max(2, r-5) (the telescoped mean of the last growth
//      factors), V_j <- s0^-j V_j, and the extension V_k = A V_{k-1} / s0 up to k = m;
//   4. Brent's minimiser of f(xi) = ||sum_k binom(m,k) (-xi/s0)^(m-k) V_k||_2^(1/m) on
//      [-sqrt(n) s0, sqrt(n) s0], each evaluation one pass over the basis;
//   5. s = s0 f(xi*) / (tol m!)^(1/m).
// 2-norms are sums of squares scaled by powers of two (exact scalings), formed per fixed chunk of rows and
// combined in a fixed order, so every block derives bit-identical L_k and f values and takes the same
// branches, and the outcome does not depend on how many CTAs run it.  Brent's scalar logic runs in
// thread 0 of every block.
#include <float.h>
#include <math.h>

#include "common.cuh"
#include "kernels.h"
#include "lowrank.cuh"
#include "select_coef.cuh"

namespace phic {

namespace {

constexpr int kMaxM = 128;

// Brent (1973, ch. 5) minimiser as a resumable state machine: after each function value it either
// names the next abscissa to evaluate (u) or finishes.  Golden-section steps into the larger part of
// the bracket, parabolic steps through the three best points when they are safe.
struct BrentSM {
  double lo, hi;        // bracket
  double x, w, v;       // best, second best, previous second best
  double fx, fw, fv;
  double step, prev;    // last step and the one before it
  double u;             // abscissa being evaluated
  double tabs;
  int evals, max_evals, started, done;
};

__host__ __device__ void brent_start(BrentSM& b, double lo, double hi, double tabs, int max_evals) {
  const double golden = 0.38196601125010515;  // (3 - sqrt 5)/2
  b.lo = lo;
  b.hi = hi;
  b.tabs = tabs;
  b.max_evals = max_evals;
  b.evals = 0;
  b.started = 0;
  b.done = 0;
  b.step = 0.0;
  b.prev = 0.0;
  b.u = lo + golden * (hi - lo);
}

__host__ __device__ void brent_feed(BrentSM& b, double fu) {
  const double golden = 0.38196601125010515;
  const double sqrt_eps = 1.4901161193847656e-08;  // sqrt(2^-52)
  b.evals += 1;
  if (!b.started) {
    b.started = 1;
    b.x = b.w = b.v = b.u;
    b.fx = b.fw = b.fv = fu;
  } else if (fu <= b.fx) {  // new best: shrink the bracket towards it
    if (b.u >= b.x) b.lo = b.x; else b.hi = b.x;
    b.v = b.w; b.fv = b.fw;
    b.w = b.x; b.fw = b.fx;
    b.x = b.u; b.fx = fu;
  } else {                  // worse: the bracket shrinks on the side of u
    if (b.u < b.x) b.lo = b.u; else b.hi = b.u;
    if (fu <= b.fw || b.w == b.x) {
      b.v = b.w; b.fv = b.fw;
      b.w = b.u; b.fw = fu;
    } else if (fu <= b.fv || b.v == b.x || b.v == b.w) {
      b.v = b.u; b.fv = fu;
    }
  }
  if (b.evals >= b.max_evals) { b.done = 1; return; }
  const double mid = 0.5 * (b.lo + b.hi);
  const double tol1 = sqrt_eps * fabs(b.x) + b.tabs / 3.0;
  const double tol2 = 2.0 * tol1;
  if (fabs(b.x - mid) <= tol2 - 0.5 * (b.hi - b.lo)) { b.done = 1; return; }
  bool parabolic = false;
  if (fabs(b.prev) > tol1) {
    // vertex of the parabola through (x,fx), (w,fw), (v,fv), as a step num/den from x
    const double r1 = (b.x - b.w) * (b.fx - b.fv);
    const double r2 = (b.x - b.v) * (b.fx - b.fw);
    double num = (b.x - b.v) * r2 - (b.x - b.w) * r1;
    double den = 2.0 * (r2 - r1);
    if (den > 0.0) num = -num; else den = -den;
    const double older = b.prev;
    b.prev = b.step;
    // accept only a step shorter than half the step before last that stays inside the bracket
    if (fabs(num) < fabs(0.5 * den * older) && num > den * (b.lo - b.x) && num < den * (b.hi - b.x)) {
      b.step = num / den;
      const double uu = b.x + b.step;
      if (uu - b.lo < tol2 || b.hi - uu < tol2) b.step = (mid >= b.x) ? tol1 : -tol1;
      parabolic = true;
    }
  }
  if (!parabolic) {
    b.prev = (b.x >= mid) ? b.lo - b.x : b.hi - b.x;
    b.step = golden * b.prev;
  }
  b.u = (fabs(b.step) >= tol1) ? b.x + b.step : b.x + (b.step > 0.0 ? tol1 : -tol1);
}

__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

struct SelShared {
  double lz[kLowRankMaxK];  // z = W^T x of a low-rank operator
  double L[kMaxM + 1];
  alignas(16) double coef[kMaxM + 1];  // read in pairs (16-byte loads) by the objective pass
  double binom[kMaxM + 1];
  double lmax, gmax, gmin, s0, inv_s0, nv, fval;
  int r, go, status;
  BrentSM br;
};

// Sums of squares over the rows are formed per fixed chunk of kChunk rows (thread t adds rows
// c kChunk + u kBlock + t, u ascending, then the block's fixed tree), and the chunks' partials are combined
// in a fixed order by every member: the result, and every decision taken on it, is the same for any team
// size.
constexpr int kChunk = kSelectChunk;
static_assert(kChunk % kBlock == 0, "a chunk is a whole number of block-wide row sweeps");

__device__ __forceinline__ int chunk_count(int n) { return (n + kChunk - 1) / kChunk; }

// Calls y = f(row) for every row of this member's chunks and stores each chunk's scaled sum of squares
// of y in part[parity][chunk].
template <typename F>
__device__ __forceinline__ void chunk_pass(int n, const Team& tm, Ssq* part, int parity, F&& f) {
  const int nch = chunk_count(n);
  for (int c = tm.rank; c < nch; c += tm.size) {
    Ssq acc = ssq_empty();
#pragma unroll
    for (int u = 0; u < kChunk / kBlock; ++u) {
      const long long row = (long long)c * kChunk + u * kBlock + threadIdx.x;
      if (row < n) ssq_add(acc, f(row));
    }
    const Ssq blk = block_ssq(acc);
    if (threadIdx.x == 0) part[(size_t)parity * nch + c] = blk;
  }
}

// Total of all chunks' partials in a fixed order; valid in thread 0.
__device__ __forceinline__ Ssq gather_chunks(const Ssq* part, int parity, int n) {
  const int nch = chunk_count(n);
  const volatile Ssq* pp = part + (size_t)parity * nch;
  Ssq acc = ssq_empty();
  for (int c = threadIdx.x; c < nch; c += kBlock) {
    Ssq x;
    x.e = pp[c].e;
    x.ssq = pp[c].ssq;
    acc = ssq_combine(acc, x);
  }
  return block_ssq(acc);
}

// The basis is stored in interleaved pairs: V_k[row] at ((k/2) n + row) 2 + k%2, so that an objective
// pass loads V_{2j} and V_{2j+1} of a row with one 16-byte load.
__device__ __forceinline__ size_t vidx(int k, int n, long long row) {
  return ((size_t)(k >> 1) * n + (size_t)row) * 2 + (k & 1);
}

// One evaluation of the objective's sum of squares: y(row) = sum_k coef_k V_k[row] (k ascending) for every
// row of this member's chunks, each chunk's scaled sum of squares of y into part[parity][chunk].  The
// rows, their order and every rounding are those of chunk_pass over the same y; the thread's kChunk/kBlock
// rows of a chunk are formed together, so that each coefficient pair is read from shared memory once (one
// 16-byte load) for all of them.  On GB300 memory instructions share the FP64 pipe's issue path: one row
// at a time took a 16-byte basis load and two 8-byte coefficient loads per two FMAs.
__device__ __forceinline__ void objective_pass(int n, int m, const Team& tm, Ssq* part, int parity,
                                               const double* __restrict__ Vb, const double* coef) {
  constexpr int U = kChunk / kBlock;
  const int nch = chunk_count(n);
  const int pairs = (m + 1) >> 1;
  const double2* __restrict__ Vp2 = reinterpret_cast<const double2*>(Vb);
  const double2* cp = reinterpret_cast<const double2*>(coef);
  for (int c = tm.rank; c < nch; c += tm.size) {
    double y[U];
#pragma unroll
    for (int u = 0; u < U; ++u) y[u] = 0.0;
    const long long row0 = (long long)c * kChunk + threadIdx.x;
    if (row0 + (U - 1) * kBlock < n) {  // every row of the thread in range (all chunks but a ragged last)
      // two pairs of basis vectors a step: 2 U independent 16-byte loads in flight a thread
      int jj = 0;
      for (; jj + 1 < pairs; jj += 2) {
        const double2 c0 = cp[jj], c1 = cp[jj + 1];
        double2 v0[U], v1[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          v0[u] = Vp2[(size_t)jj * n + (size_t)(row0 + u * kBlock)];
          v1[u] = Vp2[(size_t)(jj + 1) * n + (size_t)(row0 + u * kBlock)];
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          y[u] = fma(c0.x, v0[u].x, y[u]);
          y[u] = fma(c0.y, v0[u].y, y[u]);
          y[u] = fma(c1.x, v1[u].x, y[u]);
          y[u] = fma(c1.y, v1[u].y, y[u]);
        }
      }
      if (jj < pairs) {
        const double2 cc = cp[jj];
        double2 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = Vp2[(size_t)jj * n + (size_t)(row0 + u * kBlock)];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          y[u] = fma(cc.x, v[u].x, y[u]);
          y[u] = fma(cc.y, v[u].y, y[u]);
        }
      }
      if ((m + 1) & 1) {
#pragma unroll
        for (int u = 0; u < U; ++u) y[u] = fma(coef[m], Vb[vidx(m, n, row0 + u * kBlock)], y[u]);
      }
    } else {
      for (int jj = 0; jj < pairs; ++jj) {
        const double2 cc = cp[jj];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const long long row = row0 + u * kBlock;
          if (row < n) {
            const double2 v = Vp2[(size_t)jj * n + (size_t)row];
            y[u] = fma(cc.x, v.x, y[u]);
            y[u] = fma(cc.y, v.y, y[u]);
          }
        }
      }
      if ((m + 1) & 1) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const long long row = row0 + u * kBlock;
          if (row < n) y[u] = fma(coef[m], Vb[vidx(m, n, row)], y[u]);
        }
      }
    }
    Ssq acc = ssq_empty();
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (row0 + u * kBlock < n) ssq_add(acc, y[u]);
    const Ssq blk = block_ssq(acc);
    if (threadIdx.x == 0) part[(size_t)parity * nch + c] = blk;
  }
}

// (A x)[row] for the basis vector x = V_k (pair-interleaved, stride 2).
template <typename VT>
__device__ __forceinline__ double spmv_row(const SelectArgs& a, const VT* __restrict__ vals, const double* x, int row,
                                           int& bad) {
  const int beg = __ldg(a.rowptr + row), end = __ldg(a.rowptr + row + 1);
  double acc = 0.0;
  for (int q = beg; q < end; ++q) {
    const int col = __ldg(a.colidx + q);
    if ((unsigned)col >= (unsigned)a.n) { bad = 1; continue; }
    acc = fma((double)__ldg(vals + q), x[(size_t)col * 2], acc);
  }
  return acc;
}

}  // namespace

// Algorithm 1 on the team tm; a.part holds 2 x ceil(n / kChunk) partials and a.ctl is tm.ctl.
template <typename VT, bool LR = false>
__device__ __forceinline__ void select_body(const SelectArgs& a, Team& tm, SelShared& sh) {
  Ctl* ctl = tm.ctl;
  const int n = a.n, m = a.m;
  Ssq* part = static_cast<Ssq*>(a.part);
  const VT* __restrict__ vals = static_cast<const VT*>(a.vals);
  const long long stride = (long long)tm.size * kBlock;
  const long long first = (long long)tm.rank * kBlock + threadIdx.x;
  const bool leader = tm.rank == 0 && threadIdx.x == 0;
  int pc = 0;  // pass counter (parity of the partial buffer)
  int bad = 0;

  if (threadIdx.x == 0) {
    // max_j log binom(m, j): at the middle index (both middle indices for odd m, in the same form as
    // any j); neighbouring j differ by at least log(1 + 2/m), far above the rounding of lgamma
    double lmax = -INFINITY;
    for (int j = m / 2; j <= (m + 1) / 2; ++j) lmax = fmax(lmax, lgamma(m + 1.0) - lgamma(j + 1.0) - lgamma(m - j + 1.0));
    sh.lmax = lmax;
    sh.gmax = a.delta * log(DBL_MAX);
    sh.gmin = a.delta * log(DBL_MIN);
    sh.status = PHIC_OK;
  }

  // ---- v (given or drawn), its 2-norm; CSR structure check ------------------------------------------
  double* V0 = a.Vb;
  {
    chunk_pass(n, tm, part, pc & 1, [&](long long row) {
      if (!LR) {
        const int b0 = __ldg(a.rowptr + row), b1 = __ldg(a.rowptr + row + 1);
        if (b1 < b0 || b0 < 0 || b1 > a.nnz || (row == 0 && b0 != 0) || (row == n - 1 && b1 != a.nnz)) bad = 1;
      }
      double x;
      if (a.v) {
        x = a.v[row];
      } else {
        const double u = (double)(splitmix64_at(a.seed, (uint64_t)row) >> 11) * 0x1.0p-53;
        x = 2.0 * u - 1.0;
      }
      V0[vidx(0, n, row)] = x;
      return x;
    });
    if (__syncthreads_or(bad) && threadIdx.x == 0) set_status(ctl, PHIC_INVALID_ARG);
    if (!team_sync(tm)) return;
    const Ssq tot = gather_chunks(part, pc & 1, n);
    ++pc;
    if (threadIdx.x == 0) {
      const double lg = ssq_log_norm(tot);
      sh.nv = exp(lg);
      sh.status = read_status(ctl);
      if (sh.status == PHIC_OK && !(isfinite(lg))) sh.status = PHIC_INVALID_ARG;
    }
    __syncthreads();
    if (sh.status != PHIC_OK) {
      if (leader) {
        a.out->status = sh.status;
        set_status(ctl, sh.status);
      }
      return;
    }
  }
  // ---- V_0 = v / ||v|| and L_0 ------------------------------------------------------------------------
  {
    const double nv = sh.nv;
    chunk_pass(n, tm, part, pc & 1, [&](long long row) {
      const double x = V0[vidx(0, n, row)] / nv;
      V0[vidx(0, n, row)] = x;
      return x;
    });
    if (!team_sync(tm)) return;
    const Ssq tot = gather_chunks(part, pc & 1, n);
    ++pc;
    if (threadIdx.x == 0) {
      sh.L[0] = ssq_log_norm(tot);
      sh.r = 0;
      sh.go = 1;
    }
    __syncthreads();
  }
  // ---- guarded power basis ----------------------------------------------------------------------------
  for (int k = 1; k <= m && sh.go; ++k) {
    const double* __restrict__ Vp = a.Vb + vidx(k - 1, n, 0);
    if constexpr (LR) {
      const int r0 = (int)((long long)tm.rank * n / tm.size), r1 = (int)((long long)(tm.rank + 1) * n / tm.size);
      if (!lr_reduce(tm, static_cast<const VT*>(a.lrW), a.lr_k, 1, r0, r1,
                     [&](int row, int) { return Vp[(size_t)row * 2]; }, a.lr_part, sh.lz))
        return;
    }
    chunk_pass(n, tm, part, pc & 1, [&](long long row) {
      double y;
      if constexpr (LR) y = lr_row(static_cast<const VT*>(a.lrU), a.lr_k, (int)row, sh.lz, 1);
      else y = spmv_row<VT>(a, vals, Vp, (int)row, bad);
      a.Vb[vidx(k, n, row)] = y;
      return y;
    });
    if (__syncthreads_or(bad) && threadIdx.x == 0) set_status(ctl, PHIC_INVALID_ARG);
    if (!team_sync(tm)) return;
    const Ssq tot = gather_chunks(part, pc & 1, n);
    ++pc;
    if (threadIdx.x == 0) {
      const double Lk = ssq_log_norm(tot);
      sh.status = read_status(ctl);
      if (sh.status != PHIC_OK || Lk + 0.5 * log(k + 1.0) + sh.lmax > sh.gmax || Lk < sh.gmin || isnan(Lk)) {
        sh.go = 0;
      } else {
        sh.L[k] = Lk;
        sh.r = k;
      }
    }
    __syncthreads();
  }
  if (sh.status != PHIC_OK) {
    if (leader) a.out->status = sh.status;
    return;
  }
  const int r = sh.r;
  if (r == 0) {  // nothing accepted: xi = 0, s = 1
    if (leader) {
      a.out->xi = 0.0;
      a.out->s = 1.0;
      a.out->s0 = 0.0;
      a.out->f_star = 0.0;
      a.out->r = 0;
      a.out->evals = 0;
      a.out->status = PHIC_OK;
    }
    return;
  }
  // ---- s0 from the last growth factors; V_j <- s0^-j V_j ----------------------------------------------
  if (threadIdx.x == 0) {
    int jr = r - 5 > 2 ? r - 5 : 2;
    if (r - jr <= 0) jr = r - 1 > 0 ? r - 1 : 0;
    const double ls0 = (sh.L[r] - sh.L[jr]) / (double)(r - jr);
    sh.s0 = exp(ls0);
    sh.inv_s0 = 1.0 / sh.s0;
  }
  __syncthreads();
  if (threadIdx.x >= 1 && threadIdx.x <= r) sh.coef[threadIdx.x] = exp(-(double)threadIdx.x * log(sh.s0));  // r <= 128 < kBlock
  __syncthreads();
  for (long long row = first; row < n; row += stride)
    for (int j = 1; j <= r; ++j) a.Vb[vidx(j, n, row)] *= sh.coef[j];
  if (!team_sync(tm)) return;
  // ---- extend: V_k = A V_{k-1} / s0, k = r+1..m -------------------------------------------------------
  for (int k = r + 1; k <= m; ++k) {
    const double* __restrict__ Vp = a.Vb + vidx(k - 1, n, 0);
    const double inv_s0 = sh.inv_s0;
    if constexpr (LR) {
      const int r0 = (int)((long long)tm.rank * n / tm.size), r1 = (int)((long long)(tm.rank + 1) * n / tm.size);
      if (!lr_reduce(tm, static_cast<const VT*>(a.lrW), a.lr_k, 1, r0, r1,
                     [&](int row, int) { return Vp[(size_t)row * 2]; }, a.lr_part, sh.lz))
        return;
      for (long long row = first; row < n; row += stride)
        a.Vb[vidx(k, n, row)] = lr_row(static_cast<const VT*>(a.lrU), a.lr_k, (int)row, sh.lz, 1) * inv_s0;
    } else {
      for (long long row = first; row < n; row += stride)
        a.Vb[vidx(k, n, row)] = spmv_row<VT>(a, vals, Vp, (int)row, bad) * inv_s0;
    }
    if (!team_sync(tm)) return;
  }
  // ---- Brent on f(xi) ---------------------------------------------------------------------------------
  if (threadIdx.x == 0) {
    const double half = sqrt((double)n) * sh.s0;
    brent_start(sh.br, -half, half, 1e-8 * sh.s0, a.max_evals);
  }
  if (threadIdx.x == 0) binomial_row(m, sh.binom);
  __syncthreads();
  const double lbin = lgamma(m + 1.0);
  while (true) {
    // coefficients binom(m,k) z^(m-k), z = -u/s0
    if (threadIdx.x <= m) {
      const int kk = threadIdx.x;
      sh.coef[kk] = objective_coef(sh.binom[kk], -sh.br.u / sh.s0, m - kk);
    }
    __syncthreads();
    objective_pass(n, m, tm, part, pc & 1, a.Vb, sh.coef);  // y = sum_k coef_k V_k[row], k ascending
    if (!team_sync(tm)) return;
    const Ssq tot = gather_chunks(part, pc & 1, n);
    ++pc;
    if (threadIdx.x == 0) {
      const double lg = ssq_log_norm(tot);
      const double f = (lg == -INFINITY) ? 0.0 : exp(lg / (double)m);
      brent_feed(sh.br, f);
    }
    __syncthreads();
    if (sh.br.done) break;
  }
  if (leader) {
    const double ltm = (log(a.tol) + lbin) / (double)m;  // log (tol m!)^(1/m)
    const double s = sh.s0 * sh.br.fx / exp(ltm);
    a.out->xi = sh.br.x;
    a.out->s = s;
    a.out->s0 = sh.s0;
    a.out->f_star = sh.br.fx;
    a.out->r = r;
    a.out->evals = sh.br.evals;
    a.out->status = (isfinite(s) && isfinite(sh.br.x)) ? PHIC_OK : PHIC_NONFINITE;
  }
}

}  // namespace phic
