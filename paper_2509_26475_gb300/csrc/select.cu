// Single-instance launch of Algorithm 1: one cooperative grid, the whole grid one team.
#include "select_body.cuh"

namespace phic {

// Blocks per SM of the selection kernel: short passes (fewer blocks make the fixed-order combine and the
// barrier cheaper) against memory-level parallelism in the objective passes, which stream the basis.
// 4 blocks (64 registers): Algorithm 1 at n = 1,048,576 in 7.38 ms against 7.93 ms at 2 blocks on GB300.
#ifndef PHIC_SELECT_BLOCKS_PER_SM
#define PHIC_SELECT_BLOCKS_PER_SM 4
#endif

template <typename VT>
__global__ void __launch_bounds__(kBlock, PHIC_SELECT_BLOCKS_PER_SM) select_kernel(const SelectArgs a) {
  __shared__ SelShared sh;
  Team tm = grid_team(a.ctl, a.spin_ns);
  select_body<VT>(a, tm, sh);
}

template <typename VT>
__global__ void __launch_bounds__(kBlock) lr_select_kernel(const SelectArgs a) {
  __shared__ SelShared sh;
  Team tm = grid_team(a.ctl, a.spin_ns);
  select_body<VT, true>(a, tm, sh);
}

__global__ void params_set_kernel(phic_params* p, double xi, double s) {
  p->xi = xi;
  p->s = s;
  p->s0 = 0.0;
  p->f_star = 0.0;
  p->r = 0;
  p->evals = 0;
  p->status = PHIC_OK;
  p->pad = 0;
}

int max_select_grid() { return 4096; }


cudaError_t launch_select(const SelectArgs& a, cudaStream_t st, int* grid_out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const void* fn = a.vals_f32 ? (const void*)select_kernel<float> : (const void*)select_kernel<double>;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBlock, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorLaunchOutOfResources;
  if (per_sm > PHIC_SELECT_BLOCKS_PER_SM) per_sm = PHIC_SELECT_BLOCKS_PER_SM;
  long long need = ((long long)a.n + kSelectChunk - 1) / kSelectChunk;  // the summed passes go by chunks
  long long grid = (long long)sms * per_sm;
  if (need < grid) grid = need < 1 ? 1 : need;
  if (grid > max_select_grid()) grid = max_select_grid();
  if (grid_out) *grid_out = (int)grid;
  void* args[] = {const_cast<SelectArgs*>(&a)};
  count_launch();
  return cudaLaunchCooperativeKernel(fn, dim3((unsigned)grid), dim3(kBlock), args, 0, st);
}

cudaError_t launch_lr_select(const SelectArgs& a, cudaStream_t st) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const void* fn = a.vals_f32 ? (const void*)lr_select_kernel<float> : (const void*)lr_select_kernel<double>;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBlock, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorLaunchOutOfResources;
  if (per_sm > 2) per_sm = 2;
  long long need = ((long long)a.n + kSelectChunk - 1) / kSelectChunk;
  long long grid = (long long)sms * per_sm;
  if (need < grid) grid = need < 1 ? 1 : need;
  if (grid > kLowRankMaxGrid) grid = kLowRankMaxGrid;
  void* args[] = {const_cast<SelectArgs*>(&a)};
  count_launch();
  return cudaLaunchCooperativeKernel(fn, dim3((unsigned)grid), dim3(kBlock), args, 0, st);
}

cudaError_t launch_params_set(phic_params* p, double xi, double s, cudaStream_t st) {
  count_launch();
  params_set_kernel<<<1, 1, 0, st>>>(p, xi, s);
  return cudaGetLastError();
}

}  // namespace phic
