// Single-instance launches of Algorithm 3: one cooperative grid per phase, the whole grid one team.
#include "solve_body.cuh"

namespace phic {

template <typename T, int CW, int MINB>
__global__ void __launch_bounds__(kBlock, MINB) series_kernel(const SolveArgs a) {
  __shared__ SeriesSmem<T> sm;
  Team tm = grid_team(a.ctlS, a.spin_ns);
  int phase = 0;
  series_body<T, CW>(a, tm, sm, phase);
}

template <typename T, int CW, int MINB>
__global__ void __launch_bounds__(kBlock, MINB) recover_kernel(const SolveArgs a) {
  __shared__ RecoverSmem<T> sm;
  Team tm = grid_team(a.ctlR, a.spin_ns);
  int phase = 0;
  recover_body<T, CW>(a, tm, sm, phase, 0x7fffffff);
}

// Low-rank operators: the same bodies with A applied as U (W^T x) (one team reduction per product).
template <typename T, int CW>
__global__ void __launch_bounds__(kBlock, 2) lr_series_kernel(const SolveArgs a) {
  __shared__ SeriesSmem<T> sm;
  __shared__ LowRankSmem<T> lz;
  Team tm = grid_team(a.ctlS, a.spin_ns);
  int phase = 0;
  series_body<T, CW, true>(a, tm, sm, phase, &lz);
}

template <typename T, int CW>
__global__ void __launch_bounds__(kBlock, 2) lr_recover_kernel(const SolveArgs a) {
  __shared__ RecoverSmem<T> sm;
  __shared__ LowRankSmem<T> lz;
  Team tm = grid_team(a.ctlR, a.spin_ns);
  int phase = 0;
  recover_body<T, CW, true>(a, tm, sm, phase, 0x7fffffff, &lz);
}

// ---------------------------------------------------------------------------------------------------
namespace {

template <typename K>
cudaError_t coop_launch(K kernel, long long items, int max_per_sm, const SolveArgs& a, cudaStream_t st,
                        int* grid_out, int max_grid = 1 << 30) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlock, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorLaunchOutOfResources;
  if (per_sm > max_per_sm) per_sm = max_per_sm;
  long long need = (items + kBlock - 1) / kBlock;
  long long grid = (long long)sms * per_sm;
  if (need < grid) grid = need < 1 ? 1 : need;
  if (grid > max_grid) grid = max_grid;
  if (grid_out) *grid_out = (int)grid;
  void* args[] = {const_cast<SolveArgs*>(&a)};
  count_launch();
  return cudaLaunchCooperativeKernel((const void*)kernel, dim3((unsigned)grid), dim3(kBlock), args, 0, st);
}

template <typename T, int MINB>
cudaError_t dispatch_series_b(const SolveArgs& a, cudaStream_t st, int* g) {
  const long long items = (long long)a.n * a.S_lay.Lp2;
  const int bps = blocks_per_sm(sizeof(T));
  switch (a.S_lay.cw) {
    case 1: return coop_launch(series_kernel<T, 1, MINB>, items, bps, a, st, g);
    case 2: return coop_launch(series_kernel<T, 2, MINB>, items, bps, a, st, g);
#if PHIC_CW_MAX_F32 >= 8
    case 8:
      if constexpr (sizeof(T) == 4) return coop_launch(series_kernel<T, 8, MINB>, items, bps, a, st, g);
      return cudaErrorInvalidValue;
#endif
    default: return coop_launch(series_kernel<T, 4, MINB>, items, bps, a, st, g);
  }
}
template <typename T, int MINB>
cudaError_t dispatch_recover_b(const SolveArgs& a, cudaStream_t st, int* g) {
  const long long items = (long long)a.n * a.F_lay.Lp2;
  const int bps = blocks_per_sm(sizeof(T));
  switch (a.F_lay.cw) {
    case 1: return coop_launch(recover_kernel<T, 1, MINB>, items, bps, a, st, g);
    case 2: return coop_launch(recover_kernel<T, 2, MINB>, items, bps, a, st, g);
#if PHIC_CW_MAX_F32 >= 8
    case 8:
      if constexpr (sizeof(T) == 4) return coop_launch(recover_kernel<T, 8, MINB>, items, bps, a, st, g);
      return cudaErrorInvalidValue;
#endif
    default: return coop_launch(recover_kernel<T, 4, MINB>, items, bps, a, st, g);
  }
}
// Residency hint by tile width: 2 blocks per SM for tiles up to 4 columns, 3 for wider ones.
// Resident blocks per SM the wide-tile kernels (more than 4 columns) are built for.
#ifndef PHIC_WIDE_MINB_F32
#define PHIC_WIDE_MINB_F32 3
#endif
#ifndef PHIC_WIDE_MINB_F64
#define PHIC_WIDE_MINB_F64 3
#endif
template <typename T>
constexpr int wide_minb() { return sizeof(T) == 4 ? PHIC_WIDE_MINB_F32 : PHIC_WIDE_MINB_F64; }
template <typename T>
cudaError_t dispatch_series(const SolveArgs& a, cudaStream_t st, int* g) {
  return a.S_lay.w <= 4 ? dispatch_series_b<T, 2>(a, st, g) : dispatch_series_b<T, wide_minb<T>()>(a, st, g);
}
template <typename T>
cudaError_t dispatch_recover(const SolveArgs& a, cudaStream_t st, int* g) {
  return a.F_lay.w <= 4 ? dispatch_recover_b<T, 2>(a, st, g) : dispatch_recover_b<T, wide_minb<T>()>(a, st, g);
}
}  // namespace

template <typename T>
cudaError_t dispatch_lr_series(const SolveArgs& a, cudaStream_t st) {
  const long long items = (long long)a.n * a.S_lay.Lp2;
  const int bps = blocks_per_sm(sizeof(T)) < 2 ? blocks_per_sm(sizeof(T)) : 2;
  switch (a.S_lay.cw) {
    case 1: return coop_launch(lr_series_kernel<T, 1>, items, bps, a, st, nullptr, kLowRankMaxGrid);
    case 2: return coop_launch(lr_series_kernel<T, 2>, items, bps, a, st, nullptr, kLowRankMaxGrid);
#if PHIC_CW_MAX_F32 >= 8
    case 8:
      if constexpr (sizeof(T) == 4) return coop_launch(lr_series_kernel<T, 8>, items, bps, a, st, nullptr, kLowRankMaxGrid);
      return cudaErrorInvalidValue;
#endif
    default: return coop_launch(lr_series_kernel<T, 4>, items, bps, a, st, nullptr, kLowRankMaxGrid);
  }
}
template <typename T>
cudaError_t dispatch_lr_recover(const SolveArgs& a, cudaStream_t st) {
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

cudaError_t launch_lr_series(const SolveArgs& a, int prec, cudaStream_t st) {
  return prec == PHIC_F32 ? dispatch_lr_series<float>(a, st) : dispatch_lr_series<double>(a, st);
}
cudaError_t launch_lr_recover(const SolveArgs& a, int prec, cudaStream_t st) {
  return prec == PHIC_F32 ? dispatch_lr_recover<float>(a, st) : dispatch_lr_recover<double>(a, st);
}

cudaError_t launch_series(const SolveArgs& a, int prec, cudaStream_t st, int* grid_out) {
  return prec == PHIC_F32 ? dispatch_series<float>(a, st, grid_out) : dispatch_series<double>(a, st, grid_out);
}
cudaError_t launch_recover(const SolveArgs& a, int prec, cudaStream_t st, int* grid_out) {
  return prec == PHIC_F32 ? dispatch_recover<float>(a, st, grid_out) : dispatch_recover<double>(a, st, grid_out);
}

TileLayout pick_layout(int w, int elem_bytes) {
  const int cw_max = elem_bytes == 4 ? PHIC_CW_MAX_F32 : PHIC_CW_MAX;
  TileLayout t;
  t.w = w;
  if (cw_max >= 8 && w % 8 == 0 && w / 8 <= 32) {
    t.cw = 8;
    t.ws = w;
  } else if (cw_max >= 4 && w % 4 == 0 && w / 4 <= 32) {
    t.cw = 4;
    t.ws = w;
  } else if (cw_max >= 2 && w % 2 == 0 && w / 2 <= 32) {
    t.cw = 2;
    t.ws = w;
  } else if (w <= 32) {
    t.cw = 1;
    t.ws = w;
  } else {
    t.cw = 4;
    t.ws = (w + 3) / 4 * 4;
  }
  t.L = t.ws / t.cw;
  t.Lp2 = 1;
  while (t.Lp2 < t.L) t.Lp2 <<= 1;
  return t;
}

}  // namespace phic
