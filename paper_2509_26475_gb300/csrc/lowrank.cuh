// Matrix-free low-rank operators A = U W^T (U, W n x k, row-major): x -> U (W^T x) with O(n k) work, the
// family of large test operators of the paper's third experiment (Section 6).  Applying A to an n x w
// block X takes one team-wide reduction Z = W^T X (k x w) before the row pass.
#pragma once

#include "common.cuh"

namespace phic {

constexpr int kLowRankMaxK = PHIC_MAX_RANK;
constexpr int kLowRankMaxE = 256;   // limit on k w, the entries of Z
constexpr int kLowRankMaxGrid = 1024;

// Z = W^T X on team tm: member b reduces its rows [r0, r1) into part[b][e] (e = q w + c), the team syncs,
// and every member adds the members' partials in rank order into zs[e] (shared memory, k w doubles).
// xat(row, c) returns X(row, c) as a double; with absw the entries of W enter as |W|.  The sums are
// fixed by the team size (they are rounded per member).  Returns false if the barrier timed out.
template <typename TW, typename XF>
__device__ __forceinline__ bool lr_reduce(Team& tm, const TW* __restrict__ W, int k, int w, int r0, int r1, XF&& xat,
                                          double* part, double* zs, bool absw = false) {
  __shared__ double s_red[kBlock / 32][8];
  __shared__ double s_slice[kLowRankMaxE];
  const int E = k * w;
  double* mine = part + (size_t)tm.rank * E;
  for (int e0 = 0; e0 < E; e0 += 8) {
    double acc[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) acc[u] = 0.0;
    for (int row = r0 + (int)threadIdx.x; row < r1; row += kBlock) {
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + u;
        if (e < E) {
          const int q = e / w, c = e - q * w;
          double wv = (double)W[(size_t)row * k + q];
          if (absw) wv = fabs(wv);
          acc[u] = fma(wv, xat(row, c), acc[u]);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      double v = acc[u];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5][u] = v;
    }
    __syncthreads();
    if (threadIdx.x < 8 && e0 + (int)threadIdx.x < E) {
      double sum = 0.0;
      for (int wi = 0; wi < kBlock / 32; ++wi) sum += s_red[wi][threadIdx.x];
      mine[e0 + threadIdx.x] = sum;
    }
    __syncthreads();
  }
  if (!team_sync(tm)) return false;
  // every member: Z = sum over members in rank order; S slices of the members run side by side
  const int S = kBlock / E;  // E <= kBlock
  const int t = (int)threadIdx.x;
  if (t < S * E) {
    const int e = t % E, sl = t / E;
    double z = 0.0;
    for (int m = sl; m < tm.size; m += S) z += __ldcg(part + (size_t)m * E + e);
    s_slice[t] = z;
  }
  __syncthreads();
  if (t < E) {
    double z = 0.0;
    for (int sl = 0; sl < S; ++sl) z += s_slice[sl * E + t];
    zs[t] = z;
  }
  __syncthreads();
  return true;
}

// y = U(row, :) z for a k-vector z (shared memory, stride zstride between its entries).
template <typename TU, typename TZ>
__device__ __forceinline__ TZ lr_row(const TU* __restrict__ U, int k, int row, const TZ* z, int zstride) {
  TZ y = TZ(0);
  for (int q = 0; q < k; ++q) y = fma((TZ)U[(size_t)row * k + q], z[q * zstride], y);
  return y;
}

}  // namespace phic
