#pragma once
// Algorithm 3 of the paper (Section 4): block scaling-and-recovering truncated Taylor method for
// w_i = sum_j alpha_i^j phi_j(t_i A) v_j, i = 1..r.
//
// The two phases are device functions run by a team of CTAs (the whole grid of a single-instance launch,
// or a share of a batched launch), on one workspace:
//   series_body     -- setup (A_1 = A - xi I formed once, the reordered and scaled V), then the block
//                      series S = sum_k D_k / k! of Theorem 1 (eq. rec.D with the shift of
//                      eq. cD.shift), term by term with the truncation test (3.3).
//   recover_body    -- the first-block recovery F(:,1:r) <- A F(:,1:r) T + v0 1^T, the s-1 recovery
//                      steps of eq. rec.F.shift (Taylor series of exp(A_1 T/s) with the same test, the
//                      undo factor mu and the refresh from S), and the output w_i = F_i + alpha_i F_{r+i}.
// The data-dependent loops never return to the host: every Taylor term ends at a bounded team barrier
// inside which thread 0 of every team member reads the same team-wide norms, takes the same branch and
// publishes it to its block.  The infinity norms are maxima, so the results do not depend on the team
// size.
//
// Work split: member b of a team of G owns the contiguous rows [b n / G, (b+1) n / G) in every pass
// (balanced to one row).  Tiles are row-major: row i of an n x w block is w consecutive values at row
// stride ws (see pick_layout).  Each row is processed by L lanes of CW columns; the lanes of a row are consecutive in
// a warp, so the row sums of |x| for the infinity norm are shuffle reductions.  A thread keeps the
// same lane in every pass, so its per-column constants live in registers.
//
// GB300 cost model.  FP64 arithmetic runs at 2 FMA/clk/SM and shares its issue path with the load,
// store and shuffle instructions (one memory instruction costs about 1.25 FP64 FMA there, integer
// and FP32 work cost nothing there).  Hence:
//   - the operator is held as B = (A - xi I) 2^-eA in (column, value) pairs, one 16-byte load per
//     nonzero, with ||B||_inf < 1 (2^-eA is an exact scaling);
//   - the recovery carries G_k = B^k F_0 unscaled and F_k = c_k G_k with per-column FP64 scalars
//     c_k = (t_i 2^eA / s)^k / k! kept by thread 0, so E <- E + F_k is one FMA per element;
//   - the infinity norms that decide when a Taylor loop stops are summed in FP32 from the high words
//     of the doubles (norm_piece), with no FP64 instruction.
#include <math.h>

#include "common.cuh"
#include "kernels.h"
#include "lowrank.cuh"

// Tile shape of the block kernels: widest column chunk a lane takes (1, 2 or 4).  Two columns per lane
// with two (narrow tiles) or three (tiles of 8 or more columns) resident blocks per SM measured fastest
// on GB300 for FP64: more warps hide the gathers, and wider chunks need registers that cost residency.
#ifndef PHIC_CW_MAX
#define PHIC_CW_MAX 2
#endif
// FP32 tiles: widest column chunk, 8 floats (two 16-byte loads per gathered row): with the DIA copy of
// B a row's loads are independent, and one thread per row of 8 columns measured 15 % faster on GB300
// than two threads of 4 (46.8 vs 53.9 us per recovery term at n = 1,048,576).  One row per thread at a
// time: carrying several rows at once measured slower (the registers cost residency).
#ifndef PHIC_CW_MAX_F32
#define PHIC_CW_MAX_F32 8
#endif

namespace phic {

namespace {

// Contiguous rows of this team member and the walk over their (row, lane) items in steps of the block
// size (uniform within the block, so the shuffles always see full warps).
struct BlockRows {
  int r0, r1;
  int shift;         // log2(Lp2)
  long long padded;  // (r1 - r0) * Lp2 rounded up to a multiple of the block size
  __device__ BlockRows(int n, int Lp2, const Team& tm) {
    r0 = (int)((long long)tm.rank * n / tm.size);
    r1 = (int)((long long)(tm.rank + 1) * n / tm.size);
    shift = __ffs(Lp2) - 1;
    const long long items = (long long)(r1 - r0) << shift;
    padded = (items + kBlock - 1) / kBlock * kBlock;
  }
};

__device__ __forceinline__ void umax(unsigned long long& m, double v) {
  const unsigned long long u = dbits(v);
  m = u > m ? u : m;
}

// Per-warp maxima of two values and the bad-index / non-finite flags; thread 0 folds them into the
// team's slots inside the barrier.
struct WarpParts {
  unsigned long long a[kBlock / 32], b[kBlock / 32], c[kBlock / 32];
  int bad[kBlock / 32], nonfinite[kBlock / 32];
};

__device__ __forceinline__ void warp_parts(WarpParts& wp, unsigned long long a, unsigned long long b, int bad,
                                           int nonfinite = 0, unsigned long long c = 0) {
  a = warp_max_u64(a);
  b = warp_max_u64(b);
  c = warp_max_u64(c);
  const int anyb = __any_sync(0xffffffffu, bad);
  const int anyn = __any_sync(0xffffffffu, nonfinite);
  if ((threadIdx.x & 31) == 0) {
    wp.a[threadIdx.x >> 5] = a;
    wp.b[threadIdx.x >> 5] = b;
    wp.c[threadIdx.x >> 5] = c;
    wp.bad[threadIdx.x >> 5] = anyb;
    wp.nonfinite[threadIdx.x >> 5] = anyn;
  }
}

// Slot 2 collects the non-finite flag of a pass (as 0/1), slot 3 a third maximum (an integer).
__device__ __forceinline__ void parts_to_slots(Ctl* c, int phase, const WarpParts& wp) {
  unsigned long long a = 0, b = 0, m = 0;
  int bad = 0, nf = 0;
  for (int w = 0; w < kBlock / 32; ++w) {
    a = wp.a[w] > a ? wp.a[w] : a;
    b = wp.b[w] > b ? wp.b[w] : b;
    m = wp.c[w] > m ? wp.c[w] : m;
    bad |= wp.bad[w];
    nf |= wp.nonfinite[w];
  }
  slot_max(c, phase, 0, a);
  slot_max(c, phase, 1, b);
  if (nf) slot_max(c, phase, 2, 1ull);
  if (m) slot_max(c, phase, 3, m);
  if (bad) set_status(c, PHIC_INVALID_ARG);
}
__device__ __forceinline__ unsigned long long slot_raw(const Ctl* c, int phase, int idx) {
  return *(volatile const unsigned long long*)&c->slot[phase & 3][idx];
}

// Grid-wide norm published in a slot by the float path, back to FP64 (scaled by 2^e0).
__device__ __forceinline__ double slot_norm(const Ctl* c, int phase, int idx, int e0) {
  const unsigned long long u = *(volatile const unsigned long long*)&c->slot[phase & 3][idx];
  return ldexp((double)__int_as_float((int)(unsigned)u), e0);
}
// The same norm as the FP32 value it was summed as (scaled by 2^-e0).
__device__ __forceinline__ float slot_normf(const Ctl* c, int phase, int idx) {
  return __int_as_float((int)(unsigned)*(volatile const unsigned long long*)&c->slot[phase & 3][idx]);
}
__device__ __forceinline__ bool slot_nonfinite(const Ctl* c, int phase) {
  return *(volatile const unsigned long long*)&c->slot[phase & 3][2] != 0ull;
}
__device__ __forceinline__ void fmax_bits(unsigned long long& m, float v) {
  const unsigned long long u = (unsigned)__float_as_int(v);
  m = u > m ? u : m;
}
// bias of norm_piece for the scale 2^-e0
__device__ __forceinline__ int norm_bias(int e0) { return (896 + e0) << 20; }
__device__ __forceinline__ int scale_exponent(double ref) {
  return (ref > 0.0 && isfinite(ref)) ? ilogb(ref) : 0;
}

// Sum of products in the storage precision: fused multiply-adds.  The FP32 path can instead carry the
// products' and sums' rounding errors in a second word (error-free transformations TwoProduct by FMA and
// TwoSum; PHIC_F32_COMPENSATED=1).  With the per-step norm cap of FP32 solves (kTheta32) the rounding of
// the Taylor terms dominates and the compensation changed no error measurably (max 1.13e-6 either way
// over 128 FP32 instances against the FP64 oracle) while costing 14 % of the recovery term time, so it is
// off by default.
template <typename T>
struct DotAcc {
  T hi;
  __device__ __forceinline__ void zero() { hi = T(0); }
  __device__ __forceinline__ void add(T a, T x) { hi = fma(a, x, hi); }
  __device__ __forceinline__ T value() const { return hi; }
};
#ifndef PHIC_F32_COMPENSATED
#define PHIC_F32_COMPENSATED 0
#endif
#if PHIC_F32_COMPENSATED
template <>
struct DotAcc<float> {
  float hi, lo;
  __device__ __forceinline__ void zero() { hi = 0.f; lo = 0.f; }
  // explicitly rounded operations: a contraction into an FMA would break the error-free transformations
  __device__ __forceinline__ void add(float a, float x) {
    const float p = __fmul_rn(a, x);
    const float pe = fmaf(a, x, -p);  // exact error of the product
    const float s = __fadd_rn(hi, p);
    const float bb = __fsub_rn(s, hi);
    const float se = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));  // exact error of the sum
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(pe, se));
  }
  __device__ __forceinline__ float value() const { return __fadd_rn(hi, lo); }
};
#endif

// Entries gathered together by the CSR and ELL products: four, or two when a lane's chunk of a row is
// 32 bytes (four such gathers spilled at 80 registers a thread).
template <typename T, int CW>
constexpr int kGatherBatch = CW * sizeof(T) >= 32 ? 2 : 4;

// acc[j] = sum_q B(row, col_q) X(col_q, c0 + j) over the row's stored entries, kGatherBatch at a time so
// that their gathers are in flight together.  Columns were checked when the entries were written.
template <typename T, int CW>
__device__ __forceinline__ void spmm_ent(const int* __restrict__ rowptr, const CsrEnt<T>* __restrict__ ent,
                                         const T* __restrict__ X, int ws, int c0, int row, T (&acc)[CW]) {
  constexpr int U = kGatherBatch<T, CW>;
  const int beg = __ldg(rowptr + row), end = __ldg(rowptr + row + 1);
  DotAcc<T> d[CW];
#pragma unroll
  for (int j = 0; j < CW; ++j) d[j].zero();
  for (int q0 = beg; q0 < end; q0 += U) {
    const int cnt = end - q0;
    CsrEnt<T> e[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (u < cnt) e[u] = ent[q0 + u];
    T x[U][CW];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (u < cnt) VecIOG<T, CW>::ld(X + (size_t)e[u].col * ws + c0, x[u]);
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (u < cnt) {
#pragma unroll
        for (int j = 0; j < CW; ++j) d[j].add(e[u].v, x[u][j]);
      }
  }
#pragma unroll
  for (int j = 0; j < CW; ++j) acc[j] = d[j].value();
}

// The same over the ELL copy of B: entry q of `row` at ent[q n + row] for q < K (rows shorter than K
// padded with a zero weight on their own column), so no row bounds are loaded and the entries of
// consecutive rows are consecutive.
template <typename T, int CW>
__device__ __forceinline__ void spmm_ell_dyn(const CsrEnt<T>* __restrict__ ent, int n, int K, const T* __restrict__ X,
                                             int ws, int c0, int row, T (&acc)[CW]) {
  constexpr int U = kGatherBatch<T, CW>;
  DotAcc<T> d[CW];
#pragma unroll
  for (int j = 0; j < CW; ++j) d[j].zero();
  for (int q0 = 0; q0 < K; q0 += U) {
    CsrEnt<T> e[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (q0 + u < K) e[u] = ent[(size_t)(q0 + u) * n + row];
    T x[U][CW];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (q0 + u < K) VecIOG<T, CW>::ld(X + (size_t)e[u].col * ws + c0, x[u]);
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (q0 + u < K) {
#pragma unroll
        for (int j = 0; j < CW; ++j) d[j].add(e[u].v, x[u][j]);
      }
  }
#pragma unroll
  for (int j = 0; j < CW; ++j) acc[j] = d[j].value();
}

// The same over the DIA copy of B: the value of diagonal d (offset off[d]) in `row` at val[d n + row]
// (zero where the row has no entry on it).  The gathered rows row + off[d] follow from the offsets, so
// every load of a row is issued at once and consecutive rows read consecutive memory.  Columns outside
// [0, n) carry a zero value and are read from the row itself.
template <typename T, int CW, int D>
__device__ __forceinline__ void spmm_dia_k(const T* __restrict__ val, const int (&off)[7], int n,
                                           const T* __restrict__ X, int ws, int c0, int row, T (&acc)[CW]) {
  T v[D];
  T x[D][CW];
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const int j = row + off[d];
    const int jj = (unsigned)j < (unsigned)n ? j : row;
    v[d] = val[(size_t)d * n + row];
    VecIOG<T, CW>::ld(X + (size_t)jj * ws + c0, x[d]);
  }
  DotAcc<T> acc_d[CW];
#pragma unroll
  for (int c = 0; c < CW; ++c) acc_d[c].zero();
#pragma unroll
  for (int d = 0; d < D; ++d)
#pragma unroll
    for (int c = 0; c < CW; ++c) acc_d[c].add(v[d], x[d][c]);
#pragma unroll
  for (int c = 0; c < CW; ++c) acc[c] = acc_d[c].value();
}

template <typename T, int CW>
__device__ __forceinline__ void spmm_dia_dyn(const T* __restrict__ val, const int* off, int D, int n,
                                             const T* __restrict__ X, int ws, int c0, int row, T (&acc)[CW]) {
  DotAcc<T> acc_d[CW];
#pragma unroll
  for (int c = 0; c < CW; ++c) acc_d[c].zero();
  for (int d = 0; d < D; ++d) {
    const int j = row + off[d];
    const int jj = (unsigned)j < (unsigned)n ? j : row;
    const T v = val[(size_t)d * n + row];
    T x[CW];
    VecIOG<T, CW>::ld(X + (size_t)jj * ws + c0, x);
#pragma unroll
    for (int c = 0; c < CW; ++c) acc_d[c].add(v, x[c]);
  }
#pragma unroll
  for (int c = 0; c < CW; ++c) acc[c] = acc_d[c].value();
}

// Diagonal offsets of the DIA copy kept in registers for the widths with fixed loops (5 and 7).
struct DiaOffsets {
  int o[7];
  __device__ __forceinline__ void load(const int* off, int D) {
#pragma unroll
    for (int d = 0; d < 7; ++d) o[d] = d < D ? off[d] : 0;
  }
};

// Formats of the copy of B, as types: a row loop is instantiated once per format, so that each loop
// holds the registers of one product variant only (one loop with every variant inside spilled).
struct FmtCsr {};
struct FmtEll {};                 // run-time number of slots
template <int D> struct FmtDia {};  // D diagonals (0: run-time number)
struct FmtLowRank {};

// Operands of a row product shared by the formats.
template <typename T>
struct SpmmOps {
  const int* __restrict__ rowptr;
  const CsrEnt<T>* __restrict__ ent;
  int n, ell, ndia;
  const int* doff;  // ndia offsets (shared memory)
};

template <typename T, int CW>
__device__ __forceinline__ void spmm_fmt(FmtCsr, const SpmmOps<T>& o, const DiaOffsets&, const T* __restrict__ X,
                                         int ws, int c0, int row, T (&acc)[CW]) {
  spmm_ent<T, CW>(o.rowptr, o.ent, X, ws, c0, row, acc);
}
template <typename T, int CW>
__device__ __forceinline__ void spmm_fmt(FmtEll, const SpmmOps<T>& o, const DiaOffsets&, const T* __restrict__ X,
                                         int ws, int c0, int row, T (&acc)[CW]) {
  spmm_ell_dyn<T, CW>(o.ent, o.n, o.ell, X, ws, c0, row, acc);
}
template <typename T, int CW, int D>
__device__ __forceinline__ void spmm_fmt(FmtDia<D>, const SpmmOps<T>& o, const DiaOffsets& dor,
                                         const T* __restrict__ X, int ws, int c0, int row, T (&acc)[CW]) {
  const T* __restrict__ val = reinterpret_cast<const T*>(o.ent);
  if constexpr (D > 0) spmm_dia_k<T, CW, D>(val, dor.o, o.n, X, ws, c0, row, acc);
  else spmm_dia_dyn<T, CW>(val, o.doff, o.ndia, o.n, X, ws, c0, row, acc);
}

// Calls body(tag) with the format tag of the copy the setup built.
template <bool LR, typename Body>
__device__ __forceinline__ void with_format(int ndia, int ell, Body&& body) {
  if constexpr (LR) {
    body(FmtLowRank{});
  } else {
    if (ndia == 5) body(FmtDia<5>{});
    else if (ndia == 7) body(FmtDia<7>{});
    else if (ndia) body(FmtDia<0>{});
    else if (ell) body(FmtEll{});
    else body(FmtCsr{});
  }
}

// Where the switch on the format goes.  A Taylor loop nest runs under loop_format; each row loop in it
// runs under row_format.  With kSplit the switch encloses the whole nest, which is then instantiated
// once per format and gets a register allocation of its own (with one nest for all formats, the widest
// format's needs made the 5-diagonal loop spill its loop state: 47 against 36 us per FP32 recovery term
// at n = 1,048,576 on GB300).  Without it (kernels that run many small problems, where code size and
// build time matter more) one nest switches at every row loop: its tag is FmtAny.
struct FmtAny {};
template <typename F> constexpr bool kIsFmtAny = false;
template <> constexpr bool kIsFmtAny<FmtAny> = true;
template <bool kSplit, bool LR, typename Body>
__device__ __forceinline__ void loop_format(int ndia, int ell, Body&& body) {
  if constexpr (kSplit) with_format<LR>(ndia, ell, body);
  else body(FmtAny{});
}
template <bool LR, typename Fmt, typename Body>
__device__ __forceinline__ void row_format(Fmt f, int ndia, int ell, Body&& body) {
  if constexpr (kIsFmtAny<Fmt>) with_format<LR>(ndia, ell, body);
  else body(f);
}

// |x| 2^-e0 as an FP32 value, for the infinity-norm sums that feed the truncation test.  For a double
// the high word (sign, exponent, 20 mantissa bits) is rebiased into FP32 layout with integer
// operations (relative truncation below 2^-20; values under 2^-126 of the scale flush to 0, values above
// 2^128 saturate) so that the norms cost no FP64 instruction; Inf and NaN raise `nonfinite`.  bias
// carries (896 + e0) << 20.  An FP32 element is scaled exactly.
__device__ __forceinline__ float norm_piece(double x, int bias, float scale, int& nonfinite) {
  (void)scale;
  const int h = __double2hiint(x) & 0x7fffffff;
  nonfinite |= h >= 0x7ff00000;
  int t = h - bias;
  t = t < 0 ? 0 : t;
  t = t > 0x0FEFFFFF ? 0x0FEFFFFF : t;
  return __int_as_float(t << 3);
}
// An FP32 element is scaled exactly; Inf and NaN pass into the row sums, which the caller checks once per
// row (row_nonfinite), instead of every element here.
__device__ __forceinline__ float norm_piece(float x, int bias, float scale, int& nonfinite) {
  (void)bias;
  (void)nonfinite;
  return fabsf(x) * scale;
}
template <typename T>
__device__ __forceinline__ int row_nonfinite(float s1, float s2) {
  return sizeof(T) == 4 ? !(isfinite(s1) && isfinite(s2)) : 0;
}

// Block-level broadcast of the loop decision made by thread 0.
struct LoopCtl {
  int go;       // 1: run another term
  int k;        // index of the term to run
  int status;
  int bias;     // norm_piece bias of the current scale 2^-e0
  float fscale; // 2^-e0 as a float (FP32 tiles)
};

__device__ __forceinline__ void set_norm_scale(LoopCtl& lc, int e0) {
  lc.bias = norm_bias(e0);
  const int ef = e0 < -126 ? -126 : (e0 > 126 ? 126 : e0);
  lc.fscale = exp2f((float)-ef);
}

// Per-term column coefficients of the series, already divided by k (see series_kernel).
template <typename T>
struct SeriesTerm {
  T kd[PHIC_MAX_R], ka[PHIC_MAX_R], kt[PHIC_MAX_R];
};

// Largest per-step norm nu t / s of an FP32 solve: ln(2^24) / 2 (the FP32 rounding of the Taylor terms,
// which grow like e^(nu t / s), then stays near sqrt(u)).
constexpr double kTheta32 = 8.317766166719343;

struct SeriesScalars {
  double xi, s_used, tc[PHIC_MAX_R], cA[PHIC_MAX_R], cD[PHIC_MAX_R], cV[PHIC_MAX_R];
  int s_int, bad, eA, nodiag, ell, ndia;
  int dia_off[16];
};

// ---- scalars of the recovery steps in double-double (warp 0) --------------------------------------
// Every recovery step applies the same scalars: the Taylor coefficients c_k = (t_i 2^eA / s)^k / k! and
// the undo factor mu_i = e^(xi t_i / s).  Rounded once and reused, each would carry the same relative
// error into all s - 1 steps, and those errors would add up coherently: mu's rounding alone (its argument
// rounded, then magnified |xi t / s| times by the exponential) costs up to about |xi t| 2^-53 in the result,
// 1.6e-11 at xi t = -1.4e6 (the paper's Chebyshev example at t = 1).  Instead:
//   - c_k is formed in double-double and rounded to the tile type without bias: up with the probability
//     of the remainder's share of the gap, decided by a hash of the step, term and combination (next_coefs),
//     so that the rounding errors of different steps are independent with mean zero;
//   - the factor applied in step j is chosen so that the product of all applied factors stays within one
//     rounding of e^(j xi t / s), computed from a double-double exponent (compensated scaling).
struct DD {
  double h, l;
};
__device__ __forceinline__ DD dd_renorm(double s, double e) {
  const double h = s + e;
  return DD{h, e - (h - s)};
}
__device__ __forceinline__ DD dd_prod(double a, double b) {
  const double p = a * b;
  return DD{p, fma(a, b, -p)};
}
__device__ __forceinline__ DD dd_times(DD a, DD b) {
  const double p = a.h * b.h;
  return dd_renorm(p, fma(a.h, b.h, -p) + (a.h * b.l + a.l * b.h));
}
__device__ __forceinline__ DD dd_times_d(DD a, double b) {
  const double p = a.h * b;
  return dd_renorm(p, fma(a.h, b, -p) + a.l * b);
}
__device__ __forceinline__ DD dd_over_d(DD a, double d) {
  const double q = a.h / d;
  const double rem = fma(-q, d, a.h);  // exact remainder of the leading quotient
  return dd_renorm(q, (rem + a.l) / d);
}

// 64 uniform bits from a 64-bit key (the splitmix64 output function).
__device__ __forceinline__ unsigned long long unit_bits(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

constexpr double kLog2eHi = 1.4426950408889634, kLog2eLo = 2.0355273740931033e-17;  // 1/ln 2 in double-double

// Shared memory of the recovery is tight (one block's rows of E sit next to it at 3 blocks per SM), so the
// double-double scalars keep their leading parts in the plain arrays: tB + tBl = t_i 2^eA / s and
// c + cl = c_k; the applied product of the undo factors is (pmh + pml) 2^pe.
template <typename T>
struct RecoverScalars {
  double xi, tB[PHIC_MAX_R], tBl[PHIC_MAX_R], c[PHIC_MAX_R], cl[PHIC_MAX_R];
  double pmh[PHIC_MAX_R], pml[PHIC_MAX_R];
  int pe[PHIC_MAX_R];
  T mu_step[PHIC_MAX_R];  // the undo factor of the current step
  T coef[PHIC_MAX_R];
  T xiB;                  // -xi 2^-eA: the explicit shift of rows without a stored diagonal
  float fcoef[PHIC_MAX_R];
  T cj[PHIC_MAX_P + 1][PHIC_MAX_R];
  int s_int, series_terms, status, eA, nodiag, ell, ndia;
  int dia_off[16];
  int done, rec_init, j_done, cur;
  double cF0;
};

// Shared memory of the two bodies; a kernel that runs both keeps them in one union.
// zs / zt: Z = W^T X of a low-rank operator (FP64 sums, and scaled in the tile type).
template <typename T>
struct SeriesSmem {
  SeriesScalars sc;
  LoopCtl lc;
  SeriesTerm<T> tk;
  WarpParts wp;
};
// The recovery's loop decisions, kept by warp 0 between two barriers (in shared memory, so that none of it
// holds a register of the Taylor loop).  The truncation test compares FP32 norms scaled by 2^-e0 as the row
// sums are formed (R16): c1, c2 and nE are those scaled values.  The leader's block also keeps the counts.
struct DecideState {
  double cF;          // ||F||_inf at the start of the current step
  float c1, c2, nE;
  int status, k, e0;
  int cur_j;          // recovery step of the current Taylor loop
  int tab_k;          // coefficient table filled up to this term (see next_coefs)
  int max_inner;
  long long rec_terms;
};

template <typename T>
struct RecoverSmem {
  RecoverScalars<T> sc;
  LoopCtl lc;
  WarpParts wp;
  DecideState ds;
};
template <typename T>
struct LowRankSmem {
  double zs[kLowRankMaxE];
  T zt[kLowRankMaxE];
};

// ===================================================================================================
// Block series (Algorithm 3: setup and the first while loop)
// ===================================================================================================
// The recurrence is carried divided by k!: with X = A_1 (I kron T/s) = 2^eA B (I kron T/s),
//   V~_k = V~_{k-1} Jsh / k,   D~_k = X D~_{k-1} / k + V~_k,   S = sum_k D~_k,   c2 = ||D~_k||_inf,
// which equals the paper's D_k / k! and V_k / k! term by term but never holds the growing X^k D_1,
// which would overflow FP32 (and, for a large ||X||, FP64) long before the terms become small.
//
// Runs on the team tm; `phase` is the team's next slot phase (advanced by one per barrier).  Thread 0
// of rank 0 records the outcome in a.state (status, s_int, term count, xi, s, eA, nodiag) on every exit.
template <typename T, int CW, bool LR = false, bool kSplit = false>
__device__ __forceinline__ int series_run(const SolveArgs& a, Team& tm, SeriesSmem<T>& sm, int& phase,
                                          LowRankSmem<T>* lz = nullptr) {
  SeriesScalars& sc = sm.sc;
  LoopCtl& lc = sm.lc;
  SeriesTerm<T>& tk = sm.tk;
  WarpParts& wp = sm.wp;
  Ctl* ctl = tm.ctl;
  const int n = a.n, r = a.r, p = a.p;
  const TileLayout L = a.S_lay;

  if (threadIdx.x == 0) {
    // s <- ceil(s max|t_i|);  mu = exp((xi/s) T);  V <- V (I kron 1^T mu/s);
    // Jsh = (J kron Delta - xi I kron T)/s  (divided by s as in Algorithm 2)
    // FP32 storage uses xi rounded to FP32.  The shift is undone exactly by mu whatever its value, but
    // the diagonal a_ii - xi of B is rounded to FP32 once and then applied in every product: with xi not
    // an FP32 number, a constant diagonal makes that rounding one shift error delta on every row, which no
    // step undoes and which costs a relative delta t_i in w_i (about 1e-5 at t = 1e-4 on the 1024^2
    // advection-diffusion operator, where ulp(a_ii - xi) = 0.25).  With xi in FP32, a_ii - xi is exact
    // whenever a_ii lies within a factor 2 of xi (Sterbenz), as it does for stencil operators, whose
    // spectral centre is near their diagonal.
    const double xi = sizeof(T) == 4 ? (double)__double2float_rn(a.params->xi) : a.params->xi;
    double s = a.params->s;
    if (sizeof(T) == 4) {
      // FP32 storage: the Taylor terms of a step grow like e^(nu t / s) before they cancel, and their
      // FP32 rounding, not Algorithm 1's truncation bound, sets the error.  Keep the per-step norm
      // nu t / s at most theta_32 = ln(2^24) / 2, where nu = s0 f(xi*) is the norm estimate behind s
      // (s = nu / (tol m!)^(1/m)); FP64 steps (<= 12.8 at tol 2^-53) are below ln(2^53) / 2 already.
      const double nu = a.params->s0 * a.params->f_star;
      if (nu > 0.0 && isfinite(nu)) s = fmax(s, nu / kTheta32);
    }
    sc.s_used = s;
    int bad = !isfinite(xi) || !(s >= 0.0) || !isfinite(s);
    double tmax = 0.0;
    for (int i = 0; i < r; ++i) tmax = fmax(tmax, fabs(a.t[i]));
    double sint = ceil(s * tmax);
    if (!(sint >= 1.0)) sint = 1.0;
    if (sint > 2147483647.0) bad = 1;
    const int si = bad ? 1 : (int)sint;
    for (int i = 0; i < r; ++i) {
      sc.tc[i] = a.t[i] / si;
      sc.cA[i] = a.alpha[i] / si;
      sc.cD[i] = -(xi * a.t[i]) / si;
      sc.cV[i] = exp(xi * a.t[i] / si) / si;
    }
    sc.xi = xi;
    sc.s_int = si;
    sc.bad = bad;
    sc.eA = 0;
    sc.nodiag = 0;
    sc.ell = 0;
    sc.ndia = 0;
    lc.k = 1;
  }
  __syncthreads();
  if (sc.bad) {
    if (threadIdx.x == 0) set_status(ctl, PHIC_INVALID_ARG);
    return PHIC_INVALID_ARG;
  }
  if (a.fault && tm.rank == 0 && tm.size > 1) return PHIC_TIMEOUT;  // test hook: never arrive at the barrier

  const T* __restrict__ vals = static_cast<const T*>(a.vals);
  CsrEnt<T>* __restrict__ ent = static_cast<CsrEnt<T>*>(a.A1);
  const T* __restrict__ Vin = static_cast<const T*>(a.Vin);
  T* __restrict__ S = static_cast<T*>(a.S);
  const BlockRows br(n, L.Lp2, tm);
  const int lmask = L.Lp2 - 1;
  const int c0 = (threadIdx.x & lmask) * CW;

  T kV[CW];
  int kI[CW];
  bool kLive[CW], kUp[CW];
  const T* kSrc[CW];
#pragma unroll
  for (int j = 0; j < CW; ++j) {
    const int c = c0 + j;
    kLive[j] = c < L.w;
    const int b = kLive[j] ? c / r : 0, i = kLive[j] ? c - b * r : 0;
    kI[j] = i;
    kV[j] = (T)sc.cV[i];
    kUp[j] = kLive[j] && b >= 2;
    // column block b of V holds v0 (b = 0) or v_{p+1-b} (b >= 1): [v0, vp, ..., v1]
    kSrc[j] = !kLive[j] ? nullptr
              : (b == 0) ? (a.no_v0 ? nullptr : Vin)
                         : Vin + (size_t)(p + 1 - b - a.no_v0) * n;
  }
  int bad = 0;

  // ---- setup pass 1: CSR checks, ||A - xi I||_inf, rows without a stored diagonal -------------------
  if constexpr (!LR) {
    {
      const int ph = phase++;
      slot_reset(tm, ph);
      unsigned long long mx = 0, maxlen = 0;
      int nodiag = 0;
      // the distinct diagonal offsets (col - row) of the stored entries, as keys offset + n in a block-wide
      // hash table, then merged into the team's 16-entry table in the control block
      __shared__ int s_dkeys[32];
      __shared__ int s_dovf;
      if (threadIdx.x < 32) s_dkeys[threadIdx.x] = 0;
      if (threadIdx.x == 0) s_dovf = 0;
      __syncthreads();
      auto dia_insert = [&](int key) {
        int h = key & 31;
        for (int probe = 0; probe < 32; ++probe) {
          const int cur = *(volatile int*)&s_dkeys[h];
          if (cur == key) return;
          if (cur == 0) {
            const int old = atomicCAS(&s_dkeys[h], 0, key);
            if (old == 0 || old == key) return;
          }
          h = (h + 1) & 31;
        }
        s_dovf = 1;
      };
      for (long long it = threadIdx.x; it < br.padded; it += kBlock) {
        const int row = br.r0 + (int)(it >> br.shift), lane = (int)(it & lmask);
        if (row < br.r1 && lane == 0) {
          const int b0 = __ldg(a.rowptr + row), b1 = __ldg(a.rowptr + row + 1);
          if (b1 < b0 || b0 < 0 || b1 > a.nnz || (row == 0 && b0 != 0) || (row == n - 1 && b1 != a.nnz)) {
            bad = 1;
          } else {
            maxlen = (unsigned long long)(b1 - b0) > maxlen ? (unsigned long long)(b1 - b0) : maxlen;
            bool shifted = false;
            double rs = 0.0;
            for (int q = b0; q < b1; ++q) {
              const int col = __ldg(a.colidx + q);
              if ((unsigned)col >= (unsigned)n) { bad = 1; continue; }
              dia_insert(col - row + n);
              double v = (double)__ldg(vals + q);
              if (!shifted && col == row) {
                v -= sc.xi;
                shifted = true;
              }
              rs += fabs(v);
            }
            if (!shifted) rs += fabs(sc.xi);
            a.rowflag[row] = shifted ? 0 : 1;
            nodiag |= !shifted;
            umax(mx, rs);
          }
        }
      }
      warp_parts(wp, mx, (unsigned long long)nodiag, bad, 0, maxlen);
      __syncthreads();
      if (threadIdx.x < 32) {  // merge this block's offsets into the team's table
        const int key = s_dkeys[threadIdx.x];
        if (key != 0) {
          int h = key & 15, probe = 0;
          for (; probe < 16; ++probe) {
            const int old = atomicCAS(&ctl->dia_keys[h], 0, key);
            if (old == 0 || old == key) break;
            h = (h + 1) & 15;
          }
          if (probe == 16) atomicOr(&ctl->dia_ovf, 1);
        }
        if (threadIdx.x == 0 && s_dovf) atomicOr(&ctl->dia_ovf, 1);
      }
      if (!team_sync_lead(tm, [&] { parts_to_slots(ctl, ph, wp); },
                          [&] {
                            const double na = slot_get(ctl, ph, 0);
                            sc.eA = (na > 0.0 && isfinite(na)) ? ilogb(na) + 1 : 0;  // ||B||_inf < 1
                            sc.nodiag = slot_get(ctl, ph, 1) != 0.0;
                            // DIA copy of B when its diagonals are few and fill the rows well; else ELL
                            // when n times the longest row fits the copy's room; else CSR order
                            int nd = 0;
                            for (int q = 0; q < 16; ++q) {
                              const int key = *(volatile const int*)&ctl->dia_keys[q];
                              if (key != 0) sc.dia_off[nd++] = key - n;
                            }
                            for (int q = 1; q < nd; ++q)  // ascending offsets
                              for (int u = q; u > 0 && sc.dia_off[u - 1] > sc.dia_off[u]; --u) {
                                const int tmp = sc.dia_off[u];
                                sc.dia_off[u] = sc.dia_off[u - 1];
                                sc.dia_off[u - 1] = tmp;
                              }
                            const bool ovf = *(volatile const int*)&ctl->dia_ovf != 0;
                            const long long cells = (long long)nd * n;
                            sc.ndia = (!ovf && nd >= 1 && cells <= 2 * a.a1_cap &&
                                       cells <= (long long)a.nnz + a.nnz / 2 + 64) ? nd : 0;
                            const long long K = (long long)slot_raw(ctl, ph, 3);
                            sc.ell = (!sc.ndia && K >= 1 && K <= 64 && K * (long long)n <= a.a1_cap) ? (int)K : 0;
                            lc.status = read_status(ctl);
                          }))
        return PHIC_TIMEOUT;
    }
  } else {
    // low-rank A = U W^T: ||A - xi I||_inf <= max_i sum_q |U_iq| sum_j |W_jq| + |xi|; no stored diagonal
    const int ph = phase++;
    slot_reset(tm, ph);
    const T* __restrict__ U = static_cast<const T*>(a.lrU);
    const T* __restrict__ Wl = static_cast<const T*>(a.lrW);
    const int k = a.lr_k;
    if (!lr_reduce(tm, Wl, k, 1, br.r0, br.r1, [](int, int) { return 1.0; }, a.lr_part, lz->zs, true))
      return PHIC_TIMEOUT;
    unsigned long long mx = 0;
    for (int row = br.r0 + (int)threadIdx.x; row < br.r1; row += kBlock) {
      double rs = fabs(sc.xi);
      for (int q = 0; q < k; ++q) rs += fabs((double)U[(size_t)row * k + q]) * lz->zs[q];
      umax(mx, rs);
    }
    warp_parts(wp, mx, 1ull, 0);
    if (!team_sync_lead(tm, [&] { parts_to_slots(ctl, ph, wp); },
                        [&] {
                          const double na = slot_get(ctl, ph, 0);
                          sc.eA = (na > 0.0 && isfinite(na)) ? ilogb(na) + 1 : 0;
                          sc.nodiag = 1;  // the shift is applied to every row explicitly
                          sc.ell = 0;
                          sc.ndia = 0;
                          lc.status = read_status(ctl);
                        }))
      return PHIC_TIMEOUT;
  }
  if (lc.status != PHIC_OK) return lc.status;

  // ---- setup pass 2: entries of B = (A - xi I) 2^-eA, and k = 1: S = D = V -------------------------
  const int ph1 = phase++;
  slot_reset(tm, ph1);
  {
    const double scaleB = ldexp(1.0, -sc.eA);
    T* V1 = static_cast<T*>(a.Vt[1]);
    T* D1 = static_cast<T*>(a.Dt[1]);
    unsigned long long mx = 0;
    for (long long it = threadIdx.x; it < br.padded; it += kBlock) {
      const int row = br.r0 + (int)(it >> br.shift), lane = (int)(it & lmask);
      const bool act = row < br.r1 && lane < L.L;
      T part = T(0);
      if (act) {
        if (!LR && lane == 0 && sc.ndia) {  // DIA: per-diagonal sums in FP64, xi subtracted once
          const int b0 = __ldg(a.rowptr + row), b1 = __ldg(a.rowptr + row + 1);
          const int D = sc.ndia;
          double dsum[16];
          for (int d = 0; d < D; ++d) dsum[d] = 0.0;
          bool shifted = false;
          for (int q = b0; q < b1; ++q) {
            const int col = __ldg(a.colidx + q);
            double v = (double)__ldg(vals + q);
            if (!shifted && col == row) {
              v -= sc.xi;
              shifted = true;
            }
            int d = 0;
            while (d < D - 1 && sc.dia_off[d] != col - row) ++d;
            dsum[d] += v;
          }
          T* __restrict__ dval = reinterpret_cast<T*>(a.A1);
          for (int d = 0; d < D; ++d) dval[(size_t)d * n + row] = (T)(dsum[d] * scaleB);
        } else if (!LR && lane == 0) {
          const int b0 = __ldg(a.rowptr + row), b1 = __ldg(a.rowptr + row + 1);
          const int K = sc.ell;
          bool shifted = false;
          for (int q = b0; q < b1; ++q) {  // subtract xi once from the stored diagonal, in FP64
            const int col = __ldg(a.colidx + q);
            double v = (double)__ldg(vals + q);
            if (!shifted && col == row) {
              v -= sc.xi;
              shifted = true;
            }
            CsrEnt<T> e;
            e.col = col;
            e.v = (T)(v * scaleB);
            ent[K ? (size_t)(q - b0) * n + row : (size_t)q] = e;
          }
          for (int q = b1 - b0; q < K; ++q) {  // ELL padding: zero weight on the row's own column
            CsrEnt<T> e;
            e.col = row;
            e.v = T(0);
            ent[(size_t)q * n + row] = e;
          }
        }
        T x[CW];
#pragma unroll
        for (int j = 0; j < CW; ++j) {
          x[j] = kSrc[j] ? kSrc[j][row] * kV[j] : T(0);
          part += fabs(x[j]);
        }
        const size_t o = (size_t)row * L.ws + c0;
        VecIOG<T, CW>::st(V1 + o, x);
        VecIOG<T, CW>::st(D1 + o, x);
        VecIOG<T, CW>::st(S + o, x);
      }
      const T rs = group_sum(part, L.Lp2);
      if (act && lane == 0) umax(mx, (double)rs);
    }
    warp_parts(wp, mx, 0ull, 0);
  }

  // Loop state, meaningful in thread 0 only.
  int k = 1, status = PHIC_OK, e0 = 0;
  double c1 = INFINITY, c2 = 0.0, nS = 0.0;
  auto decide = [&]() {  // thread 0: evaluate  while c1 + c2 > tol ||S||  and prepare term k+1
    int go = 0;
    if (status == PHIC_OK && (!isfinite(c2) || !isfinite(nS))) status = PHIC_NONFINITE;  // NaN ends the test silently
    if (status == PHIC_OK && c1 + c2 > a.tol * nS) {
      if (k >= a.max_terms) status = PHIC_TERM_CAP;
      else {
        k += 1;
        c1 = c2;
        go = 1;
        const double sB = ldexp(1.0, sc.eA);
        for (int i = 0; i < r; ++i) {
          tk.kd[i] = (T)(sc.cD[i] / k);
          tk.ka[i] = (T)(sc.cA[i] / k);
          tk.kt[i] = (T)(sc.tc[i] * sB / k);
        }
      }
    }
    lc.go = go;
    lc.k = k;
    lc.status = status;
  };
  if (!team_sync_lead(tm, [&] { parts_to_slots(ctl, ph1, wp); },
                      [&] {
                        status = read_status(ctl);
                        c2 = slot_get(ctl, ph1, 0);
                        nS = c2;
                        e0 = scale_exponent(c2);  // norms of later terms are carried in FP32 scaled by 2^-e0
                        set_norm_scale(lc, e0);
                        decide();
                      }))
    return PHIC_TIMEOUT;

  // ---- k >= 2:  V <- V Jsh;  D <- A_1 D (I kron T/s) + V;  S <- S + D/k!  (divided by k!) ----------
  const T xiB = (T)(-sc.xi * ldexp(1.0, -sc.eA));  // explicit shift for rows without a stored diagonal
  const bool nodiag = sc.nodiag != 0;
  // argument fields used per row, kept in registers (the argument block may live in shared memory)
  const int* __restrict__ rowptr = a.rowptr;
  const unsigned char* __restrict__ rowflag = a.rowflag;
  const int ell = sc.ell;
  const int ndia = sc.ndia;
  DiaOffsets dor;
  dor.load(sc.dia_off, ndia);
  const SpmmOps<T> ops{rowptr, ent, n, ell, ndia, sc.dia_off};
  // the term loop per format of B (kSplit) or one loop for all (see loop_format); a barrier that times
  // out ends it with out = PHIC_TIMEOUT
  int out = PHIC_OK;
  const bool up_vec = r % CW == 0;  // FP32 tiles: a lane's columns lie in one column block (V update)
  loop_format<kSplit, LR>(ndia, ell, [&](auto lfmt) {
  while (lc.go) {
    const int kk = lc.k;
    const int ph = phase++;
    slot_reset(tm, ph);
    // this term's column coefficients: FP32 tiles keep them in registers; FP64 tiles read them from shared
    // memory where they are used (3 CW registers fewer across the product; see the V update)
    [[maybe_unused]] T kD[CW], kA[CW], kT[CW];
    if constexpr (sizeof(T) == 4) {
#pragma unroll
      for (int j = 0; j < CW; ++j) {
        kD[j] = tk.kd[kI[j]];
        kA[j] = tk.ka[kI[j]];
        kT[j] = tk.kt[kI[j]];
      }
    }
    const T* __restrict__ Vo = static_cast<const T*>(a.Vt[(kk - 1) & 1]);
    T* __restrict__ Vn = static_cast<T*>(a.Vt[kk & 1]);
    const T* __restrict__ Do = static_cast<const T*>(a.Dt[(kk - 1) & 1]);
    T* __restrict__ Dn = static_cast<T*>(a.Dt[kk & 1]);
    if constexpr (LR) {  // Z = W^T D 2^-eA for this term's products
      if (!lr_reduce(tm, static_cast<const T*>(a.lrW), a.lr_k, L.w, br.r0, br.r1,
                     [&](int row, int c) { return (double)Do[(size_t)row * L.ws + c]; }, a.lr_part, lz->zs)) {
        out = PHIC_TIMEOUT;
        return;
      }
      const double scaleB = ldexp(1.0, -sc.eA);
      for (int e = threadIdx.x; e < a.lr_k * L.w; e += kBlock) lz->zt[e] = (T)(lz->zs[e] * scaleB);
      __syncthreads();
    }
    unsigned long long mD = 0, mS = 0;
    const int bias = lc.bias;
    const float fscale = lc.fscale;
    int nf = 0;
    row_format<LR>(lfmt, ndia, ell, [&](auto fmt) {
    for (long long it = threadIdx.x; it < br.padded; it += kBlock) {
      const int row = br.r0 + (int)(it >> br.shift), lane = (int)(it & lmask);
      const bool act = row < br.r1 && lane < L.L;
      float pD = 0.f, pS = 0.f;
      if (act) {
        const size_t o = (size_t)row * L.ws + c0;
        T acc[CW];
#pragma unroll
        for (int j = 0; j < CW; ++j) acc[j] = T(0);
        if constexpr (LR) {
#pragma unroll
          for (int j = 0; j < CW; ++j)
            acc[j] = kLive[j] ? lr_row(static_cast<const T*>(a.lrU), a.lr_k, row, lz->zt + c0 + j, L.w) : T(0);
        } else {
          spmm_fmt<T, CW>(fmt, ops, dor, Do, L.ws, c0, row, acc);
        }
        if (nodiag && (LR || rowflag[row])) {  // no stored diagonal: apply the shift explicitly
          T own[CW];
          VecIOG<T, CW>::ld(Do + o, own);
#pragma unroll
          for (int j = 0; j < CW; ++j) acc[j] = fma(xiB, own[j], acc[j]);
        }
        T vo[CW], sv[CW], vn[CW], dn[CW];
        [[maybe_unused]] T vp[CW];
        VecIOG<T, CW>::ld(Vo + o, vo);
        VecIOG<T, CW>::ld(S + o, sv);
        // block b-1 of the old V, for the columns of blocks b >= 2.  FP32 tiles take it as one vector when r
        // is a multiple of the lane's width (the lane's columns then lie in one block and c0 - r is aligned),
        // which measured 9 % faster on the series; FP64 tiles read it per column in the update below (the
        // vector form measured 0.5 % slower there)
        if constexpr (sizeof(T) == 4) {
#pragma unroll
          for (int j = 0; j < CW; ++j) vp[j] = T(0);
          if (up_vec) {
            if (kUp[0]) VecIOG<T, CW>::ld(Vo + o - r, vp);
          } else {
#pragma unroll
            for (int j = 0; j < CW; ++j)
              if (kUp[j]) vp[j] = Vo[o + j - r];
          }
        }
#pragma unroll
        for (int j = 0; j < CW; ++j) {
          // block b of the new V: -xi t_i/s times block b, plus alpha_i/s times block b-1 when b >= 2
          T v;
          if constexpr (sizeof(T) == 4) {
            v = kD[j] * vo[j];
            if (kUp[j]) v = fma(kA[j], vp[j], v);
          } else {
            v = tk.kd[kI[j]] * vo[j];
            if (kUp[j]) v = fma(tk.ka[kI[j]], Vo[o + j - r], v);
          }
          const T d = fma(acc[j], sizeof(T) == 4 ? kT[j] : tk.kt[kI[j]], v);
          const T sn = sv[j] + d;
          vn[j] = kLive[j] ? v : T(0);
          dn[j] = kLive[j] ? d : T(0);
          sv[j] = kLive[j] ? sn : T(0);
          pD += norm_piece(dn[j], bias, fscale, nf);
          pS += norm_piece(sv[j], bias, fscale, nf);
        }
        VecIOG<T, CW>::st(Vn + o, vn);
        VecIOG<T, CW>::st(Dn + o, dn);
        VecIOG<T, CW>::st(S + o, sv);
        nf |= row_nonfinite<T>(pD, pS);
      }
      const float rD = group_sum(pD, L.Lp2), rS = group_sum(pS, L.Lp2);
      if (act && lane == 0) {
        fmax_bits(mD, rD);
        fmax_bits(mS, rS);
      }
    }
    });
    warp_parts(wp, mD, mS, 0, nf);
    if (!team_sync_lead(tm, [&] { parts_to_slots(ctl, ph, wp); },
                        [&] {
                          status = read_status(ctl);
                          if (status == PHIC_OK && slot_nonfinite(ctl, ph)) status = PHIC_NONFINITE;
                          c2 = slot_norm(ctl, ph, 0, e0);  // ||D_k||_inf / k!
                          nS = slot_norm(ctl, ph, 1, e0);
                          decide();
                        })) {
      out = PHIC_TIMEOUT;
      return;
    }
  }
  });
  return out != PHIC_OK ? out : lc.status;
}

template <typename T, int CW, bool LR = false, bool kSplit = false>
__device__ __forceinline__ void series_body(const SolveArgs& a, Team& tm, SeriesSmem<T>& sm, int& phase,
                                            LowRankSmem<T>* lz = nullptr) {
  int st = series_run<T, CW, LR, kSplit>(a, tm, sm, phase, lz);
  if (tm.rank == 0 && threadIdx.x == 0) {
    if (st != PHIC_OK) set_status(tm.ctl, st);
    SolveState* sv = a.state;
    sv->status = st;
    sv->s_int = sm.sc.s_int;
    sv->series_terms = sm.lc.k;
    sv->xi = sm.sc.xi;
    sv->s = sm.sc.s_used;
    sv->eA = sm.sc.eA;
    sv->nodiag = sm.sc.nodiag;
    sv->rec_init = 0;
    sv->j_done = 0;
    sv->cur = 0;
    sv->cF = 0.0;
    sv->rec_terms = 0;
    sv->max_inner = 0;
    sv->done = 0;
    sv->ell = sm.sc.ell;
    sv->ndia = sm.sc.ndia;
    for (int d = 0; d < 16; ++d) sv->dia_off[d] = d < sm.sc.ndia ? sm.sc.dia_off[d] : 0;
  }
}

// ===================================================================================================
// Recovery (Algorithm 3: first-block recovery, the for loop over j, the output)
// ===================================================================================================
// Block p of S Jt^j, column i, is sum_{a=1..p} S(:, (a, i)) (j alpha_i/s)^(p-a) / (p-a)!, because
// Jt^j = exp(j J kron Delta / s) and (J^q)[a, p] = 1 exactly when a = p - q >= 1.
template <typename T>
__device__ __forceinline__ void jt_power_coeffs(RecoverScalars<T>& rs, const SolveArgs& a, int j) {
  const int p = a.p, r = a.r;
  for (int idx = threadIdx.x; idx < p * r; idx += blockDim.x) {
    const int aa = 1 + idx / r, i = idx % r;
    const double x = (double)j * a.alpha[i] / rs.s_int;
    double c = 1.0;
    for (int q = 1; q <= p - aa; ++q) c = c * x / q;
    rs.cj[aa][i] = (T)c;
  }
}

// The undo factor of recovery step j for each combination (thread 0): the product of the factors applied
// in steps 1..j is to equal e^(j x_i), x_i = xi t_i / s.  With the applied product P = pm 2^pe (pm in
// double-double) and j x_i / ln 2 = N + f (N an integer, |f| <= 1/2, from the double-double x_i), the
// factor is 2^(N - pe) 2^f / pm rounded to the tile type; P then takes it exactly.  The product stays
// within about one rounding of e^(j x_i) whatever j is.  Where that target leaves the double range (the
// factor or the product underflows), the plain e^(x_i) of the paper is applied.  Run by the lanes of
// warp 0, lane i for combination i.
// The table entry of a coefficient c (double-double): its nearest value in T, the neighbour on the side of
// the remainder and the probability of rounding to that neighbour, as a 32-bit threshold.
template <typename T>
__device__ __forceinline__ CoefEntry<T> coef_entry(DD c);
template <>
__device__ __forceinline__ CoefEntry<double> coef_entry<double>(DD c) {
  CoefEntry<double> e{c.h, c.l, c.h, c.h, 0u, (float)c.h};
  if (c.l != 0.0 && isfinite(c.h)) {
    e.alt = nextafter(c.h, c.l > 0.0 ? INFINITY : -INFINITY);
    e.thr = (unsigned)fmin(c.l / (e.alt - c.h) * 4294967296.0, 4294967295.0);
  }
  return e;
}
template <>
__device__ __forceinline__ CoefEntry<float> coef_entry<float>(DD c) {
  const float f = __double2float_rn(c.h);
  CoefEntry<float> e{c.h, c.l, f, f, 0u, f};
  if (isfinite(f)) {
    const double rem = (c.h - (double)f) + c.l;  // c - f (the first difference is exact)
    if (rem != 0.0) {
      e.alt = nextafterf(f, rem > 0.0 ? INFINITY : -INFINITY);
      e.thr = (unsigned)fmin(rem / ((double)e.alt - (double)f) * 4294967296.0, 4294967295.0);
    }
  }
  return e;
}

// c_k of recovery step j for every combination, rounded to the tile type without bias: up with the
// probability of the remainder's share of the gap, decided by a hash of (j, k, i), so that the rounding
// errors of different steps are independent with mean zero.  Run by the lanes of warp 0, lane i for
// combination i.  The double-double recursion c_k = c_(k-1) (t_i 2^eA / s) / k runs only the first time a
// step reaches k (tab_k: terms already in the table); later steps read the table and round with integer
// operations (on GB300 each FP64 instruction of one lane costs the FP64 pipe a whole warp's time, and this
// sits between every two Taylor terms).  Out of line, so that the Taylor loop keeps its registers.
// c_k of combination i from c_(k-1) (in sc.c, sc.cl) by the double-double recursion, entered in the table
// when k <= kCoefTab: the first time a step reaches k (out of line: it runs rarely, and the Taylor loop keeps
// its registers).
template <typename T>
__device__ __noinline__ CoefEntry<T> coef_new(RecoverScalars<T>& sc, CoefEntry<T>* __restrict__ tab, int i, int k) {
  const DD tBd{sc.tB[i], sc.tBl[i]};
  const DD cd = k == 1 ? tBd : dd_over_d(dd_times(DD{sc.c[i], sc.cl[i]}, tBd), (double)k);
  const CoefEntry<T> e = coef_entry<T>(cd);
  if (k <= kCoefTab) tab[(size_t)(k - 1) * PHIC_MAX_R + i] = e;
  return e;
}

// pf: the entry of (k, lane) when the caller loaded it already (pf_ok), see prefetch_coef.
template <typename T>
__device__ __forceinline__ void next_coefs(RecoverScalars<T>& sc, CoefEntry<T>* __restrict__ tab, int tab_k, int r,
                                           int k, int j, const CoefEntry<T>& pf, bool pf_ok) {
  const int i = threadIdx.x & 31;
  if (i >= r) return;  // r <= PHIC_MAX_R < 32: one combination per lane
  CoefEntry<T> e;
  if (pf_ok) {
    e = pf;
  } else if (k <= tab_k) {
    e = tab[(size_t)(k - 1) * PHIC_MAX_R + i];
  } else {
    e = coef_new(sc, tab, i, k);
  }
  sc.c[i] = e.ch;
  sc.cl[i] = e.cl;
  const unsigned long long key = ((unsigned long long)j << 32) ^ ((unsigned long long)k << 8) ^ (unsigned long long)i;
  sc.coef[i] = (unsigned)(unit_bits(key) >> 32) < e.thr ? e.alt : e.base;
  sc.fcoef[i] = e.fcoef;
}

// The table entry of term k for this lane's combination, if the table has it (loaded while the team
// barrier waits; next_coefs takes it from the register).
template <typename T>
__device__ __forceinline__ bool prefetch_coef(const CoefEntry<T>* __restrict__ tab, int tab_k, int r, int k,
                                              CoefEntry<T>& pf) {
  const int i = threadIdx.x & 31;
  if (k > tab_k || i >= r) return false;
  pf = tab[(size_t)(k - 1) * PHIC_MAX_R + i];
  return true;
}

template <typename T>
__device__ __noinline__ void undo_factors(RecoverScalars<T>& sc, const double* t, int r, int j) {
  for (int i = threadIdx.x & 31; i < r; i += 32) {
    const DD x = dd_over_d(dd_prod(sc.xi, t[i]), (double)sc.s_int);  // x_i = xi t_i / s
    const DD y = dd_times(dd_times_d(x, (double)j), DD{kLog2eHi, kLog2eLo});
    const double N = rint(y.h);
    const T plain = (T)exp(x.h);  // the paper's e^(x_i), for targets outside the double range
    sc.mu_step[i] = plain;
    if (!(fabs(N) < 1e6)) continue;
    const double f = (y.h - N) + y.l;
    const double ph = sc.pmh[i], pl = sc.pml[i];
    double q = exp2(f) / ph;
    q -= q * (pl / ph);
    const double mu = ldexp(q, (int)N - sc.pe[i]);
    const T muT = (T)mu;
    const DD np = dd_times_d(DD{ph, pl}, (double)muT);
    if (!(muT != T(0)) || !isfinite(mu) || !(np.h != 0.0) || !isfinite(np.h)) continue;
    int ex = 0;
    sc.pmh[i] = frexp(np.h, &ex);
    sc.pml[i] = ldexp(np.l, -ex);
    sc.pe[i] += ex;
    sc.mu_step[i] = muT;
  }
}

// Recovery step j: F_k = A_1 F_{k-1} T / (s k) is carried as F_k = c_k G_k with G_k = B G_{k-1},
// G_0 = F and c_k = c_{k-1} t_i 2^eA / (s k) per column, so that E <- E + F_k is fma(c_k, G_k, E).
//
// Runs on the team tm from the state the series left (or a previous slice recorded) and performs at most
// max_steps outer steps j; it writes the output once j reaches s_int - 1, and otherwise records in
// a.state where the next slice resumes.  Returns 1 once the solve is finished (output written or an
// error recorded).
//
// E, the sum of one step's terms, is private to a step and to the rows of each team member: with e_sm
// (shared memory of at least e_bytes) a member whose rows fit keeps its E there, off DRAM and L2.
template <typename T, int CW, bool LR = false, bool kSplit = false>
__device__ __forceinline__ int recover_body(const SolveArgs& a, Team& tm, RecoverSmem<T>& sm, int& phase,
                                            int max_steps, LowRankSmem<T>* lz = nullptr, T* e_sm = nullptr,
                                            unsigned e_bytes = 0) {
  RecoverScalars<T>& sc = sm.sc;
  LoopCtl& lc = sm.lc;
  WarpParts& wp = sm.wp;
  Ctl* ctl = tm.ctl;
  const int n = a.n, r = a.r, p = a.p;
  const TileLayout L = a.F_lay;
  const int ws_s = a.S_lay.ws;
  const volatile SolveState* vs = a.state;

  if (threadIdx.x == 0) {
    sc.status = vs->status;
    if (sc.status == PHIC_OK) sc.status = read_status(a.ctlS);
    sc.s_int = vs->s_int;
    sc.series_terms = vs->series_terms;
    sc.xi = vs->xi;
    sc.eA = vs->eA;
    sc.xiB = (T)(-vs->xi * ldexp(1.0, -vs->eA));
    sc.nodiag = vs->nodiag;
    sc.ell = vs->ell;
    sc.ndia = vs->ndia;
    for (int d = 0; d < 16; ++d) sc.dia_off[d] = vs->dia_off[d];
    sc.done = vs->done;
    sc.rec_init = vs->rec_init;
    sc.j_done = vs->j_done;
    sc.cur = vs->cur;
    sc.cF0 = vs->cF;
    if (sc.status == PHIC_OK) {
      const double sB = ldexp(1.0, sc.eA);
      for (int i = 0; i < r; ++i) {
        const DD tBd = dd_over_d(DD{a.t[i] * sB, 0.0}, (double)sc.s_int);  // T <- I_2 kron T/s, times 2^eA for B
        sc.tB[i] = tBd.h;
        sc.tBl[i] = tBd.l;
        if (sc.rec_init) {  // a later slice: the product of the undo factors applied so far
          sc.pmh[i] = vs->pm_h[i];
          sc.pml[i] = vs->pm_l[i];
          sc.pe[i] = vs->pe[i];
        } else {
          sc.pmh[i] = 1.0;
          sc.pml[i] = 0.0;
          sc.pe[i] = 0;
        }
      }
    }
  }
  __syncthreads();
  if (sc.done) return 1;  // finished in an earlier launch
  const bool leader = tm.rank == 0 && threadIdx.x == 0;
  DecideState& ds = sm.ds;
  if (threadIdx.x == 0) {
    ds.status = PHIC_OK;
    ds.k = 0;
    ds.e0 = 0;
    ds.cur_j = 0;
    ds.tab_k = sc.rec_init ? vs->coef_k : 0;
    ds.cF = sc.cF0;
    ds.c1 = ds.c2 = ds.nE = 0.f;
    ds.rec_terms = vs->rec_terms;
    ds.max_inner = vs->max_inner;
  }
  __syncthreads();
  auto finish = [&](int st) {
    if (leader) {
      const long long rec_terms = ds.rec_terms;
      const int max_inner = ds.max_inner;
      if (st != PHIC_OK) set_status(ctl, st);
      const int s1 = read_status(a.ctlS);
      int fin = s1 != PHIC_OK ? s1 : read_status(ctl);
      if (fin == PHIC_OK) fin = st;
      SolveState* sw = a.state;
      sw->done = 1;
      sw->rec_terms = rec_terms;
      sw->max_inner = max_inner;
      if (a.stats) {
        a.stats->status = fin;
        a.stats->s_int = sc.s_int;
        a.stats->series_terms = sc.series_terms;
        a.stats->max_inner_terms = max_inner;
        a.stats->recovery_terms = rec_terms;
        a.stats->spmm_count = (long long)(sc.series_terms - 1) + 1 + rec_terms;
        a.stats->xi = sc.xi;
        a.stats->s = vs->s;
        a.stats->op_format = LR ? PHIC_OP_LOWRANK : sc.ndia ? PHIC_OP_DIA : sc.ell ? PHIC_OP_ELL : PHIC_OP_CSR;
        a.stats->op_slots = LR ? 0 : sc.ndia ? sc.ndia : sc.ell;
      }
    }
  };
  if (sc.status != PHIC_OK) {
    finish(sc.status);
    return 1;
  }

  const T* __restrict__ vals = static_cast<const T*>(a.vals);
  const CsrEnt<T>* __restrict__ ent = static_cast<const CsrEnt<T>*>(a.A1);
  const T* __restrict__ S = static_cast<const T*>(a.S);
  const T* __restrict__ Vin = static_cast<const T*>(a.Vin);
  const BlockRows br(n, L.Lp2, tm);
  const int lmask = L.Lp2 - 1;
  const int c0 = (threadIdx.x & lmask) * CW;
  // E of this member's rows, in shared memory when they fit (every thread reads back only the elements it
  // wrote, so no barrier orders them).  Either way row `row` is at E + row ws: for shared memory E is
  // the generic address br.r0 rows before the buffer, so that the loops index both cases alike and every
  // access they make lies inside it.
  const bool e_local = e_sm != nullptr && (size_t)(br.r1 - br.r0) * L.ws * sizeof(T) <= e_bytes;
  T* __restrict__ E = e_local ? reinterpret_cast<T*>(reinterpret_cast<uintptr_t>(e_sm) -
                                                     (uintptr_t)br.r0 * L.ws * sizeof(T))
                              : static_cast<T*>(a.E);
  // per-column facts of this thread's lane, computed where used (so that none of them stays live across
  // the Taylor loop): column c0 + j is live when below w; block p of F when at least r; combination i
  auto col_live = [&](int j) { return c0 + j < L.w; };
  auto col_blkp = [&](int j) { return c0 + j < L.w && c0 + j >= r; };
  auto col_i = [&](int j) { const int c = c0 + j; return c >= L.w ? 0 : (c < r ? c : c - r); };
  int bad = 0;

  CoefEntry<T>* __restrict__ ctab = static_cast<CoefEntry<T>*>(a.coeftab);
  int cur = sc.cur;

  // ---- F = S(:, [blk 0, blk p]);  F(:,1:r) <- A F(:,1:r) T + v0 1^T (unshifted A, t undivided) -----
  if (!sc.rec_init) {
    if constexpr (LR) {  // Z = W^T S(:, blk 0) for the unshifted product A F(:, 1:r)
      if (!lr_reduce(tm, static_cast<const T*>(a.lrW), a.lr_k, r, br.r0, br.r1,
                     [&](int row, int c) { return (double)S[(size_t)row * ws_s + c]; }, a.lr_part, lz->zs)) {
        finish(PHIC_TIMEOUT);
        return 1;
      }
      for (int e = threadIdx.x; e < a.lr_k * r; e += kBlock) lz->zt[e] = (T)lz->zs[e];
      __syncthreads();
    }
    const int ph = phase++;
    slot_reset(tm, ph);
    T* F = static_cast<T*>(a.Ft[0]);
    const T* v0 = a.no_v0 ? nullptr : Vin;
    unsigned long long mx = 0;
    for (long long it = threadIdx.x; it < br.padded; it += kBlock) {
      const int row = br.r0 + (int)(it >> br.shift), lane = (int)(it & lmask);
      const bool act = row < br.r1 && lane < L.L;
      T part = T(0);
      if (act) {
        T f[CW];
#pragma unroll
        for (int j = 0; j < CW; ++j) {
          T v = T(0);
          if (col_live(j) && !col_blkp(j)) {
            const int i = col_i(j);
            T acc = T(0);
            if constexpr (LR) {
              acc = lr_row(static_cast<const T*>(a.lrU), a.lr_k, row, lz->zt + i, r);
            } else {
              const int beg = __ldg(a.rowptr + row), end = __ldg(a.rowptr + row + 1);
              for (int q = beg; q < end; ++q) {
                const int col = __ldg(a.colidx + q);
                if ((unsigned)col >= (unsigned)n) { bad = 1; continue; }
                acc = fma(__ldg(vals + q), S[(size_t)col * ws_s + i], acc);
              }
            }
            v = fma(acc, (T)a.t[i], v0 ? v0[row] : T(0));
          } else if (col_blkp(j)) {
            v = S[(size_t)row * ws_s + p * r + col_i(j)];
          }
          f[j] = v;
          part += fabs(v);
        }
        VecIOG<T, CW>::st(F + (size_t)row * L.ws + c0, f);
      }
      const T rs = group_sum(part, L.Lp2);
      if (act && lane == 0) umax(mx, (double)rs);
    }
    warp_parts(wp, mx, 0ull, bad);
    cur = 0;
    if (!team_sync_lead_w(tm, [] {}, [&] { parts_to_slots(ctl, ph, wp); },
                          [&] {
                            const int st = read_status(ctl);
                            const double f = slot_get(ctl, ph, 0);
                            __syncwarp();
                            if (threadIdx.x == 0) {
                              ds.status = st;
                              ds.cF = f;
                              lc.status = st;
                            }
                          })) {
      finish(PHIC_TIMEOUT);
      return 1;
    }
  } else if (threadIdx.x == 0) {
    lc.status = PHIC_OK;
  }
  __syncthreads();
  const bool nodiag = sc.nodiag != 0;
  // argument fields used per row, kept in registers (the argument block may live in shared memory)
  const int* __restrict__ rowptr = a.rowptr;
  const unsigned char* __restrict__ rowflag = a.rowflag;
  // tol in FP32 for the test on the scaled norms (a tol below the FP32 range stops no loop before max_terms,
  // as a tol of 0 would not)
  const float tolf = (float)(a.tol > 0x1.0p-125 ? a.tol : 0x1.0p-125);
  const int max_terms = a.max_terms;
  const int ell = sc.ell;
  const int ndia = sc.ndia;
  DiaOffsets dor;
  dor.load(sc.dia_off, ndia);
  const SpmmOps<T> ops{rowptr, ent, n, ell, ndia, sc.dia_off};

  // E = F; k = 0; c1 = inf; c2 = ||F||;  while c1 + c2 > tol ||E||: next term.  Run by every lane of warp 0
  // on its own copy d of the state (identical in all lanes); lane 0 stores it back.
  auto decide = [&](DecideState& d, const CoefEntry<T>& pf, bool pf_ok) {
    int go = 0;
    if (d.status == PHIC_OK && (!isfinite(d.c2) || !isfinite(d.nE))) d.status = PHIC_NONFINITE;
    if (d.status == PHIC_OK && d.c1 + d.c2 > tolf * d.nE) {
      if (d.k >= max_terms) d.status = PHIC_TERM_CAP;
      else {
        d.k += 1;
        d.c1 = d.c2;
        go = 1;
        next_coefs(sc, ctab, d.tab_k, r, d.k, d.cur_j, pf, pf_ok);
        if (d.k > d.tab_k && d.k <= kCoefTab) d.tab_k = d.k;
      }
    }
    __syncwarp();
    if (threadIdx.x == 0) {
      ds = d;
      lc.go = go;
      lc.k = d.k;
      lc.status = d.status;
    }
  };

  // ---- for j = 1 : s-1 ------------------------------------------------------------------------------
  const int j_first = sc.j_done + 1;
  const long long j_stop = (long long)sc.j_done + (long long)max_steps;
  int jstep = j_first;
  // the loop over j per format of B (kSplit) or one loop for all (see loop_format); a barrier that times
  // out ends it with timed_out
  bool timed_out = false;
  loop_format<kSplit, LR>(ndia, ell, [&](auto lfmt) {
  for (; jstep <= sc.s_int - 1 && jstep <= j_stop && lc.status == PHIC_OK; ++jstep) {
    if (threadIdx.x < 32) {
      DecideState d = ds;
      d.k = 0;
      d.cur_j = jstep;
      d.e0 = scale_exponent(d.cF);  // norms of this step's terms are carried in FP32 scaled by 2^-e0
      d.c1 = INFINITY;
      d.c2 = (float)ldexp(d.cF, -d.e0);
      d.nE = d.c2;
      if (threadIdx.x == 0) set_norm_scale(lc, d.e0);
      decide(d, CoefEntry<T>{}, false);
    }
    __syncthreads();
    while (lc.go) {
      const int kk = lc.k;
      const int ph = phase++;
      slot_reset(tm, ph);
      // this term's coefficients of the lane's columns: FP32 tiles keep them in registers; FP64 tiles read
      // them from shared memory where they are used (below)
      [[maybe_unused]] T kC[CW];
      [[maybe_unused]] float kF[CW];
      if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int j = 0; j < CW; ++j) {
          kC[j] = col_live(j) ? sc.coef[col_i(j)] : T(0);
          kF[j] = col_live(j) ? sc.fcoef[col_i(j)] : 0.f;
        }
      }
      const T* __restrict__ Go = static_cast<const T*>(a.Ft[cur]);
      T* __restrict__ Gn = static_cast<T*>(a.Ft[cur ^ 1]);
      if constexpr (LR) {  // Z = W^T G 2^-eA for this term's products
        if (!lr_reduce(tm, static_cast<const T*>(a.lrW), a.lr_k, L.w, br.r0, br.r1,
                       [&](int row, int c) { return (double)Go[(size_t)row * L.ws + c]; }, a.lr_part, lz->zs)) {
          timed_out = true;
          return;
        }
        const double scaleB = ldexp(1.0, -sc.eA);
        for (int e = threadIdx.x; e < a.lr_k * L.w; e += kBlock) lz->zt[e] = (T)(lz->zs[e] * scaleB);
        __syncthreads();
      }
      unsigned long long mF = 0, mE = 0;
      const int bias = lc.bias;
      const float fscale = lc.fscale;
      int nf = 0;
      row_format<LR>(lfmt, ndia, ell, [&](auto fmt) {
      for (long long it = threadIdx.x; it < br.padded; it += kBlock) {
        const int row = br.r0 + (int)(it >> br.shift), lane = (int)(it & lmask);
        const bool act = row < br.r1 && lane < L.L;
        float pF = 0.f, pE = 0.f;
        if (act) {
          T acc[CW];
          if constexpr (LR) {
#pragma unroll
            for (int j = 0; j < CW; ++j)
              acc[j] = col_live(j) ? lr_row(static_cast<const T*>(a.lrU), a.lr_k, row, lz->zt + c0 + j, L.w) : T(0);
          } else {
            spmm_fmt<T, CW>(fmt, ops, dor, Go, L.ws, c0, row, acc);
          }
          const size_t o = (size_t)row * L.ws + c0;
          const bool shift_row = nodiag && (LR || rowflag[row]);
          T e[CW];
          if (kk == 1 || shift_row) {
            T own[CW];
            VecIOG<T, CW>::ld(Go + o, own);
            if (shift_row) {
#pragma unroll
              for (int j = 0; j < CW; ++j) acc[j] = fma(sc.xiB, own[j], acc[j]);
            }
            if (kk == 1) {
#pragma unroll
              for (int j = 0; j < CW; ++j) e[j] = own[j];  // E = F at the start of the step
            }
          }
          if (kk != 1) VecIO<T, CW>::ld(E + o, e);
#pragma unroll
          for (int j = 0; j < CW; ++j) {
            // F_k = c_k G_k;  E <- E + F_k.  In FP64 the coefficients are read from shared memory here rather
            // than held in registers across the row loop: 12 registers fewer in the product's live range (at
            // 80 registers the loop spilled state that it reloaded from local memory every row; 1024^2
            // recovery 354.7 -> 350.8 ms on GB300).  FP32 runs at 128 registers without spills, and the
            // reads cost it 12 %.
            T ck;
            float fk;
            if constexpr (sizeof(T) == 8) {
              ck = col_live(j) ? sc.coef[col_i(j)] : T(0);
              fk = col_live(j) ? sc.fcoef[col_i(j)] : 0.f;
            } else {
              ck = kC[j];
              fk = kF[j];
            }
            e[j] = fma(ck, acc[j], e[j]);
            pF += fk * norm_piece(acc[j], bias, fscale, nf);
            pE += norm_piece(e[j], bias, fscale, nf);
          }
          VecIOG<T, CW>::st(Gn + o, acc);
          VecIO<T, CW>::st(E + o, e);
          nf |= row_nonfinite<T>(pF, pE);
        }
        const float rF = group_sum(pF, L.Lp2), rE = group_sum(pE, L.Lp2);
        if (act && lane == 0) {
          fmax_bits(mF, rF);
          fmax_bits(mE, rE);
        }
      }
      });
      warp_parts(wp, mF, mE, 0, nf);
      cur ^= 1;
      CoefEntry<T> pf;  // the next term's coefficient entry of this lane, loaded while the barrier waits
      bool pf_ok = false;
      if (!team_sync_lead_w(tm, [&] { pf_ok = prefetch_coef(ctab, ds.tab_k, r, ds.k + 1, pf); },
                            [&] { parts_to_slots(ctl, ph, wp); },
                            [&] {
                              DecideState d = ds;
                              d.status = read_status(ctl);
                              if (d.status == PHIC_OK && slot_nonfinite(ctl, ph)) d.status = PHIC_NONFINITE;
                              d.c2 = slot_normf(ctl, ph, 0);
                              d.nE = slot_normf(ctl, ph, 1);
                              decide(d, pf, pf_ok);
                            })) {
        timed_out = true;
        return;
      }
    }
    if (leader) {
      ds.rec_terms += lc.k;
      ds.max_inner = lc.k > ds.max_inner ? lc.k : ds.max_inner;
    }
    if (lc.status != PHIC_OK) break;

    // ---- E <- E mu;  S <- S Jt;  F <- E + S(:, [blk 0, blk p]);  F(:,1:r) <- E(:,1:r) -------------
    const int ph = phase++;
    slot_reset(tm, ph);
    jt_power_coeffs(sc, a, jstep);
    if (threadIdx.x < 32) undo_factors(sc, a.t, r, jstep);
    __syncthreads();
    {
      T* __restrict__ F = static_cast<T*>(a.Ft[cur]);
      unsigned long long mx = 0;
      for (long long it = threadIdx.x; it < br.padded; it += kBlock) {
        const int row = br.r0 + (int)(it >> br.shift), lane = (int)(it & lmask);
        const bool act = row < br.r1 && lane < L.L;
        T part = T(0);
        if (act) {
          const size_t o = (size_t)row * L.ws + c0;
          T e[CW];
          VecIO<T, CW>::ld(E + o, e);
#pragma unroll
          for (int j = 0; j < CW; ++j) {
            T v = col_live(j) ? e[j] * sc.mu_step[col_i(j)] : T(0);
            if (col_blkp(j)) {
              const int i = col_i(j);
              const T* srow = S + (size_t)row * ws_s;
              for (int aa = 1; aa <= p; ++aa) v = fma(srow[aa * r + i], sc.cj[aa][i], v);
            }
            e[j] = col_live(j) ? v : T(0);
            part += fabs(e[j]);
          }
          VecIOG<T, CW>::st(F + o, e);
        }
        const T rs = group_sum(part, L.Lp2);
        if (act && lane == 0) umax(mx, (double)rs);
      }
      warp_parts(wp, mx, 0ull, 0);
      if (!team_sync_lead_w(tm, [] {}, [&] { parts_to_slots(ctl, ph, wp); },
                            [&] {
                              const double f = slot_get(ctl, ph, 0);
                              const int st = read_status(ctl);
                              __syncwarp();
                              if (threadIdx.x == 0) {
                                ds.cF = f;
                                ds.status = st;
                                lc.status = st;
                              }
                            })) {
        timed_out = true;
        return;
      }
    }
  }
  });
  if (timed_out) {
    finish(PHIC_TIMEOUT);
    return 1;
  }

  if (lc.status == PHIC_OK && jstep <= sc.s_int - 1) {
    // slice ends between outer steps: record where the next one resumes
    if (leader) {
      SolveState* sw = a.state;
      sw->rec_init = 1;
      sw->j_done = jstep - 1;
      sw->coef_k = ds.tab_k;
      for (int i = 0; i < r; ++i) {
        sw->pm_h[i] = sc.pmh[i];
        sw->pm_l[i] = sc.pml[i];
        sw->pe[i] = sc.pe[i];
      }
      sw->cur = cur;
      sw->cF = ds.cF;
      sw->rec_terms = ds.rec_terms;
      sw->max_inner = ds.max_inner;
    }
    return 0;
  }

  // ---- w_i = F(:, i) + alpha_i F(:, r+i)   (p = 0: w_i = F(:, i) = exp(t_i A) v0) -------------------
  if (lc.status == PHIC_OK) {
    const T* __restrict__ F = static_cast<const T*>(a.Ft[cur]);
    T* __restrict__ W = static_cast<T*>(a.W);
    const long long total = (long long)n * r;
    const long long stride = (long long)tm.size * kBlock;
    for (long long idx = (long long)tm.rank * kBlock + threadIdx.x; idx < total; idx += stride) {
      const int i = (int)(idx / n), row = (int)(idx - (long long)i * n);
      const T* frow = F + (size_t)row * L.ws;
      W[idx] = (p == 0) ? frow[i] : fma((T)a.alpha[i], frow[r + i], frow[i]);
    }
  }
  finish(lc.status);
  return 1;
}

}  // namespace
}  // namespace phic
