// Single-instance launches of Algorithm 3, series phase (and the tile layout): one cooperative grid,
// the whole grid one team.  The recovery phase is in recover.cu.
#include "coop_launch.cuh"

namespace phic {

template <typename T, int CW, int MINB>
__global__ void __launch_bounds__(kBlock, MINB) series_kernel(const SolveArgs a) {
  __shared__ SeriesSmem<T> sm;
  Team tm = grid_team(a.ctlS, a.spin_ns);
  int phase = 0;
  series_body<T, CW, false, true>(a, tm, sm, phase);
}

// Low-rank operators: the same body with A applied as U (W^T x) (one team reduction per product).
template <typename T, int CW>
__global__ void __launch_bounds__(kBlock, 2) lr_series_kernel(const SolveArgs a) {
  __shared__ SeriesSmem<T> sm;
  __shared__ LowRankSmem<T> lz;
  Team tm = grid_team(a.ctlS, a.spin_ns);
  int phase = 0;
  series_body<T, CW, true>(a, tm, sm, phase, &lz);
}

namespace {

// Resident blocks per SM a series kernel is built for: 2 for tiles up to 4 columns; for wider tiles
// PHIC_SERIES_MINB_F32 when FP32 lanes hold at most 4 floats (their loops fit 64 registers: 5.98 ->
// 5.22 ms per 28-term series at n = 1,048,576 on GB300), else wide_minb.
#ifndef PHIC_SERIES_MINB_F32
#define PHIC_SERIES_MINB_F32 4
#endif
#ifndef PHIC_SERIES_MINB_ODD_F64
#define PHIC_SERIES_MINB_ODD_F64 2
#endif
#ifndef PHIC_SERIES_MINB_F32_CW5
#define PHIC_SERIES_MINB_F32_CW5 3
#endif
template <typename T, int CW, bool kWide>
constexpr int series_minb() {
  return !kWide ? 2
         : (sizeof(T) == 4 && CW <= 4)     ? PHIC_SERIES_MINB_F32
         : (sizeof(T) == 4 && CW == 5)     ? PHIC_SERIES_MINB_F32_CW5
         : (CW == 3 || CW == 5)            ? PHIC_SERIES_MINB_ODD_F64
                                           : wide_minb<T>();
}

template <typename T, bool kWide>
cudaError_t dispatch_series_b(const SolveArgs& a, cudaStream_t st, int* g) {
  const long long items = (long long)a.n * a.S_lay.Lp2;
  const int bps = blocks_per_sm(sizeof(T));
  switch (a.S_lay.cw) {
    case 1: return coop_launch(series_kernel<T, 1, series_minb<T, 1, kWide>()>, items, bps, a, st, g);
    case 2: return coop_launch(series_kernel<T, 2, series_minb<T, 2, kWide>()>, items, bps, a, st, g);
#if PHIC_CW_MAX_F32 >= 8
    case 8:
      if constexpr (sizeof(T) == 4)
        return coop_launch(series_kernel<T, 8, series_minb<T, 8, kWide>()>, items, bps, a, st, g);
      return cudaErrorInvalidValue;
#endif
    case 3:
    case 5:
      if constexpr (kWide) {
        if (a.S_lay.cw == 3) return coop_launch(series_kernel<T, 3, series_minb<T, 3, kWide>()>, items, bps, a, st, g);
        return coop_launch(series_kernel<T, 5, series_minb<T, 5, kWide>()>, items, bps, a, st, g);
      }
      return cudaErrorInvalidValue;
    default: return coop_launch(series_kernel<T, 4, series_minb<T, 4, kWide>()>, items, bps, a, st, g);
  }
}
template <typename T>
cudaError_t dispatch_series(const SolveArgs& a, cudaStream_t st, int* g) {
  return a.S_lay.w <= 4 ? dispatch_series_b<T, false>(a, st, g) : dispatch_series_b<T, true>(a, st, g);
}
}  // namespace

template <typename T>
cudaError_t dispatch_lr_series(const SolveArgs& a, cudaStream_t st) {
  const long long items = (long long)a.n * a.S_lay.Lp2;
  const int bps = blocks_per_sm(sizeof(T)) < 2 ? blocks_per_sm(sizeof(T)) : 2;
  switch (a.S_lay.cw) {
    case 1: return coop_launch(lr_series_kernel<T, 1>, items, bps, a, st, nullptr, kLowRankMaxGrid);
    case 2: return coop_launch(lr_series_kernel<T, 2>, items, bps, a, st, nullptr, kLowRankMaxGrid);
    case 3:
    case 5:  // FP64 tiles whose width divides by 3 or 5 (solve_layout)
      if constexpr (sizeof(T) == 8) {
        if (a.S_lay.cw == 3) return coop_launch(lr_series_kernel<T, 3>, items, bps, a, st, nullptr, kLowRankMaxGrid);
        return coop_launch(lr_series_kernel<T, 5>, items, bps, a, st, nullptr, kLowRankMaxGrid);
      }
      return cudaErrorInvalidValue;
#if PHIC_CW_MAX_F32 >= 8
    case 8:
      if constexpr (sizeof(T) == 4) return coop_launch(lr_series_kernel<T, 8>, items, bps, a, st, nullptr, kLowRankMaxGrid);
      return cudaErrorInvalidValue;
#endif
    default: return coop_launch(lr_series_kernel<T, 4>, items, bps, a, st, nullptr, kLowRankMaxGrid);
  }
}
cudaError_t launch_lr_series(const SolveArgs& a, int prec, cudaStream_t st) {
  return prec == PHIC_F32 ? dispatch_lr_series<float>(a, st) : dispatch_lr_series<double>(a, st);
}
cudaError_t launch_series(const SolveArgs& a, int prec, cudaStream_t st, int* grid_out) {
  return prec == PHIC_F32 ? dispatch_series<float>(a, st, grid_out) : dispatch_series<double>(a, st, grid_out);
}
// Odd widths from 3 to 31 columns are padded by one column (computed as zero), so that a lane carries
// two or more values with vector loads, and a row needs half the lanes.
#ifndef PHIC_PAD_ODD
#define PHIC_PAD_ODD 1
#endif

// FP64 tiles of at least this many columns take 4 columns per lane when their width allows (1024²
// recovery, 8 columns: 105.7 -> 98.9 us per term on GB300; a 4-column tile on one lane per row was
// slower, 19.6 -> 21.9 us at 64^3).
#ifndef PHIC_WIDE_CW4_F64
#define PHIC_WIDE_CW4_F64 8
#endif

#ifndef PHIC_ODD_CW_F32
#define PHIC_ODD_CW_F32 1
#endif
TileLayout pick_layout(int w, int elem_bytes, bool odd_cw) {
  const int wp = (PHIC_PAD_ODD && w >= 3 && w < 32 && (w & 1)) ? w + 1 : w;
  const int cw_max = elem_bytes == 4 ? PHIC_CW_MAX_F32 : (wp >= PHIC_WIDE_CW4_F64 && wp % 4 == 0 ? 4 : PHIC_CW_MAX);
  TileLayout t;
  t.w = w;
  if (cw_max >= 8 && wp % 8 == 0 && wp / 8 <= 32) {
    t.cw = 8;
    t.ws = wp;
  } else if (cw_max >= 4 && wp % 4 == 0 && wp / 4 <= 32) {
    t.cw = 4;
    t.ws = wp;
  } else if (cw_max >= 2 && wp % 2 == 0 && wp / 2 <= 32) {
    t.cw = 2;
    t.ws = wp;
  } else if (wp <= 32) {
    t.cw = 1;
    t.ws = wp;
  } else {
    t.cw = 4;
    t.ws = (w + 3) / 4 * 4;
  }
  t.L = t.ws / t.cw;
  t.Lp2 = 1;
  while (t.Lp2 < t.L) t.Lp2 <<= 1;
  // The lanes of a row are padded to a power of two, and an idle lane costs its warp's instructions all
  // the same (in FP64 a whole FP64 instruction): where 3 or 5 columns a lane fill a row's lanes better,
  // take them.  The 1024^2 series, 20 columns: 4 columns a lane use 8 lanes for 5 live ones, 5 a lane use
  // 4 of 4 (GB300, 54 terms: FP64 29.8 -> 20.0 ms; FP32 at 28 terms 4.55 -> 4.15 ms).
  if (odd_cw && (elem_bytes == 8 || PHIC_ODD_CW_F32) && w > 4) {
    for (const int cw : {5, 3}) {
      if (w % cw != 0 || w / cw > 32) continue;
      int lp2 = 1;
      while (lp2 < w / cw) lp2 <<= 1;
      if (lp2 * cw < t.Lp2 * t.cw) {
        t.cw = cw;
        t.ws = w;
        t.L = w / cw;
        t.Lp2 = lp2;
      }
    }
  }
  return t;
}

}  // namespace phic
