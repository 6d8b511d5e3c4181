#pragma once
// Single-instance kernels of Algorithm 3's recovery phase and their launch (one cooperative grid, the
// whole grid one team), as templates: recover_f32.cu and recover_f64.cu instantiate one precision each,
// so that the two compile side by side.
#include "coop_launch.cuh"

namespace phic {

extern __shared__ __align__(16) unsigned char recover_dyn_smem[];

// The dynamic shared memory the block was launched with, for E (see recover_body).
__device__ __forceinline__ unsigned dynamic_smem_bytes() {
  unsigned b;
  asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(b));
  return b;
}

template <typename T, int CW, int MINB>
__global__ void __launch_bounds__(kBlock, MINB) recover_kernel(const SolveArgs a) {
  __shared__ RecoverSmem<T> sm;
  Team tm = grid_team(a.ctlR, a.spin_ns);
  int phase = 0;
  const unsigned eb = dynamic_smem_bytes();
  recover_body<T, CW, false, true>(a, tm, sm, phase, 0x7fffffff, nullptr,
                                   eb ? reinterpret_cast<T*>(recover_dyn_smem) : nullptr, eb);
}

// Low-rank operators: the same body with A applied as U (W^T x) (one team reduction per product).
template <typename T, int CW>
__global__ void __launch_bounds__(kBlock, 2) lr_recover_kernel(const SolveArgs a) {
  __shared__ RecoverSmem<T> sm;
  __shared__ LowRankSmem<T> lz;
  Team tm = grid_team(a.ctlR, a.spin_ns);
  int phase = 0;
  recover_body<T, CW, true>(a, tm, sm, phase, 0x7fffffff, &lz);
}

namespace {

// Keeping the recovery's E in shared memory (recover_body) takes two of the four tile passes of every
// Taylor term off DRAM and L2.  The dynamic shared memory a launch of `kernel` at b blocks per SM
// needs for one block's rows of E, if they fit next to its static shared memory; 0 otherwise.
#ifndef PHIC_E_SMEM
#define PHIC_E_SMEM 1
#endif
template <typename K>
size_t e_smem_bytes(K kernel, const SolveArgs& a, size_t elem, int b) {
  if (!PHIC_E_SMEM || b < 1) return 0;
  int dev = 0, sms = 0, optin = 0, sm_total = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sm_total, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess)
    return 0;
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) return 0;
  long long grid = (long long)sms * b;
  const long long need = ((long long)a.n * a.F_lay.Lp2 + kBlock - 1) / kBlock;
  if (need < grid) grid = need < 1 ? 1 : need;
  const long long rows = (a.n + grid - 1) / grid;  // the most rows a team member owns
  const size_t bytes = ((size_t)rows * a.F_lay.ws * elem + 15) / 16 * 16;
  const size_t reserve = 1024;  // shared memory the hardware keeps per block
  if (bytes > (size_t)optin || (size_t)b * (bytes + fa.sharedSizeBytes + reserve) > (size_t)sm_total) return 0;
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess) return 0;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kBlock, bytes) != cudaSuccess || occ < b) return 0;
  return bytes;
}

// Resident blocks per SM of the recovery kernel for tiles wider than 4 columns.  FP64: wide_minb (3).
// FP32: 2, with 128 registers: at 3 blocks (80 registers) the loop nest reloaded spilled state from
// local memory, 2.5 loads a warp-row that missed L1 (shared memory holds E there); at 2 blocks the
// 1024^2 recovery (E in shared memory either way) runs 2882 terms in 58.5 against 74.7 ms on GB300.
#ifndef PHIC_RECOVER_MINB_F32
#define PHIC_RECOVER_MINB_F32 2
#endif
template <typename T>
constexpr int recover_wide_minb() {
  return sizeof(T) == 4 ? PHIC_RECOVER_MINB_F32 : wide_minb<T>();
}

// Tiles up to 4 columns: the 2-block kernel.  Wider tiles: the recover_wide_minb kernel with E in shared
// memory if it fits at that residency, else the 2-block kernel (128 registers) at 2 blocks per SM with
// E in shared memory if it fits there, else the recover_wide_minb kernel with E in the workspace.
template <typename T, int CW>
cudaError_t launch_recover_cw(const SolveArgs& a, cudaStream_t st, int* g) {
  constexpr int WB = recover_wide_minb<T>();
  const long long items = (long long)a.n * a.F_lay.Lp2;
  const int cap = blocks_per_sm(sizeof(T));
  auto k2 = recover_kernel<T, CW, 2>;
  const int b2 = cap < 2 ? cap : 2;
  if (a.F_lay.w <= 4) return coop_launch(k2, items, b2, a, st, g, 1 << 30, e_smem_bytes(k2, a, sizeof(T), b2));
  auto kw = recover_kernel<T, CW, WB>;
  const int bw = cap < WB ? cap : WB;
  if (const size_t d = e_smem_bytes(kw, a, sizeof(T), bw)) return coop_launch(kw, items, bw, a, st, g, 1 << 30, d);
  if (const size_t d = e_smem_bytes(k2, a, sizeof(T), b2)) return coop_launch(k2, items, b2, a, st, g, 1 << 30, d);
  return coop_launch(kw, items, bw, a, st, g);
}

template <typename T>
cudaError_t dispatch_recover(const SolveArgs& a, cudaStream_t st, int* g) {
  switch (a.F_lay.cw) {
    case 1: return launch_recover_cw<T, 1>(a, st, g);
    case 2: return launch_recover_cw<T, 2>(a, st, g);
#if PHIC_CW_MAX_F32 >= 8
    case 8:
      if constexpr (sizeof(T) == 4) return launch_recover_cw<T, 8>(a, st, g);
      return cudaErrorInvalidValue;
#endif
    default: return launch_recover_cw<T, 4>(a, st, g);
  }
}
}  // namespace

template <typename T>
inline cudaError_t dispatch_lr_recover(const SolveArgs& a, cudaStream_t st) {
  const long long items = (long long)a.n * a.F_lay.Lp2;
  const int bps = blocks_per_sm(sizeof(T)) < 2 ? blocks_per_sm(sizeof(T)) : 2;
  switch (a.F_lay.cw) {
    case 1: return coop_launch(lr_recover_kernel<T, 1>, items, bps, a, st, nullptr, kLowRankMaxGrid);
    case 2: return coop_launch(lr_recover_kernel<T, 2>, items, bps, a, st, nullptr, kLowRankMaxGrid);
#if PHIC_CW_MAX_F32 >= 8
    case 8:
      if constexpr (sizeof(T) == 4) return coop_launch(lr_recover_kernel<T, 8>, items, bps, a, st, nullptr, kLowRankMaxGrid);
      return cudaErrorInvalidValue;
#endif
    default: return coop_launch(lr_recover_kernel<T, 4>, items, bps, a, st, nullptr, kLowRankMaxGrid);
  }
}

}  // namespace phic
