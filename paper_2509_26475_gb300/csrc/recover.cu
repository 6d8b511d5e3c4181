// Single-instance launches of Algorithm 3, recovery phase: one cooperative grid, the whole grid one team.
#include "coop_launch.cuh"

namespace phic {

template <typename T, int CW, int MINB>
__global__ void __launch_bounds__(kBlock, MINB) recover_kernel(const SolveArgs a) {
  __shared__ RecoverSmem<T> sm;
  Team tm = grid_team(a.ctlR, a.spin_ns);
  int phase = 0;
  recover_body<T, CW, false, true>(a, tm, sm, phase, 0x7fffffff);
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
template <typename T>
cudaError_t dispatch_recover(const SolveArgs& a, cudaStream_t st, int* g) {
  return a.F_lay.w <= 4 ? dispatch_recover_b<T, 2>(a, st, g) : dispatch_recover_b<T, wide_minb<T>()>(a, st, g);
}
}  // namespace

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

cudaError_t launch_lr_recover(const SolveArgs& a, int prec, cudaStream_t st) {
  return prec == PHIC_F32 ? dispatch_lr_recover<float>(a, st) : dispatch_lr_recover<double>(a, st);
}

cudaError_t launch_recover(const SolveArgs& a, int prec, cudaStream_t st, int* grid_out) {
  return prec == PHIC_F32 ? dispatch_recover<float>(a, st, grid_out) : dispatch_recover<double>(a, st, grid_out);
}

}  // namespace phic
