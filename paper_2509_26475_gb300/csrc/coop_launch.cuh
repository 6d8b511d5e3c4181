#pragma once
// Cooperative launch of a single-instance kernel: the whole grid is one team, sized to what stays
// resident (at most max_per_sm blocks per SM, and no more blocks than the rows need).
#include "solve_body.cuh"

namespace phic {

// dyn_smem bytes of dynamic shared memory per block (the kernel's attribute is raised to allow them).
template <typename K>
inline cudaError_t coop_launch(K kernel, long long items, int max_per_sm, const SolveArgs& a, cudaStream_t st,
                               int* grid_out, int max_grid = 1 << 30, size_t dyn_smem = 0) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  if (dyn_smem > 0) {
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_smem);
    if (e != cudaSuccess) return e;
  }
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlock, dyn_smem);
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
  return cudaLaunchCooperativeKernel((const void*)kernel, dim3((unsigned)grid), dim3(kBlock), args, dyn_smem, st);
}

// Residency the kernels are built for: 2 blocks per SM for tiles up to 4 columns; for wider tiles the
// value below (3 measured fastest on GB300 for both precisions).
#ifndef PHIC_WIDE_MINB_F32
#define PHIC_WIDE_MINB_F32 3
#endif
#ifndef PHIC_WIDE_MINB_F64
#define PHIC_WIDE_MINB_F64 3
#endif
template <typename T>
constexpr int wide_minb() { return sizeof(T) == 4 ? PHIC_WIDE_MINB_F32 : PHIC_WIDE_MINB_F64; }
}  // namespace phic
