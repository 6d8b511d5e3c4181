#pragma once
// Coefficients of Algorithm 1's objective (Section 3): f(xi) = ||sum_k binom(m,k) z^(m-k) V_k||^(1/m) with
// z = -xi/s0.  Near its minimum the sum cancels heavily, so every coefficient is formed with one
// rounding of an exact (or doubly-precise) value: binom(m, k) in 128-bit integers, z^e in double-double.
// Used by the selection kernels and by the coefficient test hook of the C ABI.
#include <math.h>

namespace phic {

// (ah, al) <- (ah + al)(bh + bl) in double-double arithmetic: Dekker's exact product through an FMA, then
// a fast two-sum.  An overflowing leading product is returned as it is (+-inf).
__device__ __forceinline__ void dd_mul(double& ah, double& al, double bh, double bl) {
  const double p = ah * bh;
  if (!isfinite(p)) {
    ah = p;
    al = 0.0;
    return;
  }
  const double e = fma(ah, bh, -p) + (ah * bl + al * bh);
  const double s = p + e;
  al = e - (s - p);
  ah = s;
}

// z^e for an integer e >= 0 by binary exponentiation (square and multiply) carried in double-double and
// rounded once: within about an ulp of the exact power, in at most 2 log2(e) double-double products.
__device__ __forceinline__ double pow_int(double z, int e) {
  double rh = 1.0, rl = 0.0, bh = z, bl = 0.0;
  while (e > 0) {
    if (e & 1) dd_mul(rh, rl, bh, bl);
    e >>= 1;
    if (e) dd_mul(bh, bl, bh, bl);
  }
  return isfinite(rh) ? rh + rl : rh;
}

// binom(m, k) for k = 0..m (m <= 128) in exact 128-bit integer arithmetic, each rounded once to double.
__device__ __forceinline__ void binomial_row(int m, double* out) {
  unsigned __int128 c = 1;
  out[0] = 1.0;
  for (int k = 1; k <= m; ++k) {
    const unsigned __int128 num = (unsigned __int128)(m - k + 1), den = (unsigned __int128)k;
    const unsigned __int128 q = c / den, rem = c % den;
    c = q * num + rem * num / den;  // c num / den without overflow (c num is divisible by den)
    out[k] = (double)c;
  }
}

// binom(m, k) z^(m-k) from the rounded binomial and the once-rounded power: one more rounding.
__device__ __forceinline__ double objective_coef(double binom_mk, double z, int e) {
  return binom_mk * pow_int(z, e);
}

}  // namespace phic
