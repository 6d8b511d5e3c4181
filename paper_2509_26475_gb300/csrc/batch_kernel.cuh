#pragma once
// Many independent instances of the method in one persistent cooperative launch.
//
// Each instance is run by a team of CTAs with the same bodies as the single-instance kernels
// (Algorithm 1, then the series and the recovery of Algorithm 3), synchronised by a bounded barrier on
// the instance's own control block, so teams never wait for one another.  The host planner decides the
// team sizes and which CTAs form each team; every CTA walks its list of (instance, rank) entries in the
// planner's global instance order, which rules out circular waits while all CTAs are resident (the
// cooperative launch guarantees that).  An instance's description is copied into shared memory before
// its team starts on it; precision and lane width are dispatched at run time, so FP64 and FP32
// instances of any width share the launch.
#include "select_body.cuh"
#include "solve_body.cuh"

namespace phic {

namespace {

union BatchSmem {
  SeriesSmem<double> s64;
  SeriesSmem<float> s32;
  RecoverSmem<double> r64;
  RecoverSmem<float> r32;
  SelShared sel;
};

// Every body is a separate (not inlined) function, so each keeps the register allocation it has in its
// own kernel instead of sharing one allocation for the union of all paths.
template <typename T, int CW>
__device__ __noinline__ void series_call(const SolveArgs& a, Team& tm, SeriesSmem<T>& sm, int& phase) {
  series_body<T, CW>(a, tm, sm, phase);
}
template <typename T, int CW>
__device__ __noinline__ void recover_call(const SolveArgs& a, Team& tm, RecoverSmem<T>& sm, int& phase, int steps) {
  recover_body<T, CW>(a, tm, sm, phase, steps);
}
template <typename VT>
__device__ __noinline__ void select_call(const SelectArgs& a, Team& tm, SelShared& sh) {
  select_body<VT>(a, tm, sh);
}

template <typename T>
__device__ __forceinline__ void run_series(const SolveArgs& a, Team& tm, BatchSmem& u, int& phase);
// Lane widths follow pick_layout: FP64 tiles take 1, 2 or 4 columns per lane, FP32 tiles 1, 2, 4 or 8,
// and FP64 series tiles whose width divides by 3 or 5 that many where it leaves no idle lanes (batched
// and served FP32 instances keep the power-of-two lanes: two more bodies per kernel took the build of
// each batched translation unit from 85 to 136 s, for lanes that are not bound by the FP64 pipe).
template <>
__device__ __forceinline__ void run_series<double>(const SolveArgs& a, Team& tm, BatchSmem& u, int& phase) {
  if (a.S_lay.cw == 1) series_call<double, 1>(a, tm, u.s64, phase);
  else if (a.S_lay.cw == 2) series_call<double, 2>(a, tm, u.s64, phase);
  else if (a.S_lay.cw == 3) series_call<double, 3>(a, tm, u.s64, phase);
  else if (a.S_lay.cw == 5) series_call<double, 5>(a, tm, u.s64, phase);
  else series_call<double, 4>(a, tm, u.s64, phase);
}
template <>
__device__ __forceinline__ void run_series<float>(const SolveArgs& a, Team& tm, BatchSmem& u, int& phase) {
  if (a.S_lay.cw == 1) series_call<float, 1>(a, tm, u.s32, phase);
  else if (a.S_lay.cw == 2) series_call<float, 2>(a, tm, u.s32, phase);
#if PHIC_CW_MAX_F32 >= 8
  else if (a.S_lay.cw == 8) series_call<float, 8>(a, tm, u.s32, phase);
#endif
  else series_call<float, 4>(a, tm, u.s32, phase);
}

template <typename T>
__device__ __forceinline__ void run_recover(const SolveArgs& a, Team& tm, BatchSmem& u, int& phase, int steps);
template <>
__device__ __forceinline__ void run_recover<double>(const SolveArgs& a, Team& tm, BatchSmem& u, int& phase,
                                                     int steps) {
  if (a.F_lay.cw == 1) recover_call<double, 1>(a, tm, u.r64, phase, steps);
  else if (a.F_lay.cw == 2) recover_call<double, 2>(a, tm, u.r64, phase, steps);
  else recover_call<double, 4>(a, tm, u.r64, phase, steps);
}
template <>
__device__ __forceinline__ void run_recover<float>(const SolveArgs& a, Team& tm, BatchSmem& u, int& phase,
                                                    int steps) {
  if (a.F_lay.cw == 1) recover_call<float, 1>(a, tm, u.r32, phase, steps);
  else if (a.F_lay.cw == 2) recover_call<float, 2>(a, tm, u.r32, phase, steps);
#if PHIC_CW_MAX_F32 >= 8
  else if (a.F_lay.cw == 8) recover_call<float, 8>(a, tm, u.r32, phase, steps);
#endif
  else recover_call<float, 4>(a, tm, u.r32, phase, steps);
}

template <typename T>
__device__ __forceinline__ void run_instance(const BatchInst& bi, Team& tm, BatchSmem& u) {
  int phase = 0;
  if (bi.phases & kPhaseSelect) {
    if (bi.sel.vals_f32) select_call<float>(bi.sel, tm, u.sel);
    else select_call<double>(bi.sel, tm, u.sel);
    if (!team_sync(tm)) return;  // the parameters are read by every member below
  }
  if (bi.phases & kPhaseSeries) {
    run_series<T>(bi.sa, tm, u, phase);
    if (!team_sync(tm)) return;  // the series state is read by every member below
  }
  if (bi.phases & kPhaseRecover) run_recover<T>(bi.sa, tm, u, phase, bi.max_steps);
}

}  // namespace

template <int MINB>
__global__ void __launch_bounds__(kBlock, MINB) batch_kernel(const BatchArgs b) {
  __shared__ BatchSmem u;
  __shared__ BatchInst bi;
  const int e0 = b.sched_ptr[blockIdx.x], e1 = b.sched_ptr[blockIdx.x + 1];
  for (int e = e0; e < e1; ++e) {
    const SchedEntry se = b.sched[e];
    __syncthreads();  // the previous instance is done with the shared copies
    {
      const int4* src = reinterpret_cast<const int4*>(b.inst + se.inst);
      int4* dst = reinterpret_cast<int4*>(&bi);
      for (int q = threadIdx.x; q < (int)(sizeof(BatchInst) / sizeof(int4)); q += kBlock) dst[q] = src[q];
    }
    __syncthreads();
    Team tm{bi.sa.ctlR, se.rank, bi.team, b.spin_ns, 0ull};
    if (bi.prec == PHIC_F32) run_instance<float>(bi, tm, u);
    else run_instance<double>(bi, tm, u);
  }
}

static_assert(sizeof(BatchInst) % sizeof(int4) == 0, "BatchInst is copied in 16-byte words");

template <int MINB>
int batch_occupancy_of() {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<MINB>, kBlock, 0) != cudaSuccess) return 0;
  return per_sm;
}

template <int MINB>
cudaError_t launch_batch_of(const BatchArgs& b, int grid, cudaStream_t st) {
  void* args[] = {const_cast<BatchArgs*>(&b)};
  count_launch();
  return cudaLaunchCooperativeKernel((const void*)batch_kernel<MINB>, dim3((unsigned)grid), dim3(kBlock), args, 0, st);
}

}  // namespace phic
