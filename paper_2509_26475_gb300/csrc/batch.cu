// Batched kernel for two resident blocks per SM (up to 128 registers per thread) and the dispatch.
#include "batch_kernel.cuh"

namespace phic {

int batch_occupancy_minb3();
cudaError_t launch_batch_minb3(const BatchArgs& b, int grid, cudaStream_t st);

int batch_occupancy(int minb) { return minb >= 3 ? batch_occupancy_minb3() : batch_occupancy_of<2>(); }

cudaError_t launch_batch(const BatchArgs& b, int grid, int minb, cudaStream_t st) {
  return minb >= 3 ? launch_batch_minb3(b, grid, st) : launch_batch_of<2>(b, grid, st);
}

namespace {
__global__ void batch_pending_kernel(const BatchInst* inst, int count, int* out) {
  __shared__ int total;
  if (threadIdx.x == 0) total = 0;
  __syncthreads();
  int mine = 0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) {
    const BatchInst& b = inst[i];
    if ((b.phases & (kPhaseSeries | kPhaseRecover)) == 0) continue;
    const volatile SolveState* st = b.sa.state;
    mine += st->done ? 0 : 1;
  }
  atomicAdd(&total, mine);
  __syncthreads();
  if (threadIdx.x == 0) *out = total;
}
__global__ void batch_collect_kernel(const BatchInst* inst, int count, int* done, phic_stats* stats,
                                     phic_params* params) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= count) return;
  const BatchInst& b = inst[k];
  const bool solve = (b.phases & (kPhaseSeries | kPhaseRecover)) != 0;
  done[k] = solve ? ((const volatile SolveState*)b.sa.state)->done : 1;
  if (solve && b.sa.stats) stats[k] = *b.sa.stats;
  const phic_params* prm = solve ? b.sa.params : b.sel.out;
  if (prm) params[k] = *prm;
}
}  // namespace

cudaError_t launch_batch_collect(const BatchInst* inst, int count, int* done, phic_stats* stats, phic_params* params,
                                 cudaStream_t st) {
  if (count < 1) return cudaSuccess;
  count_launch();
  batch_collect_kernel<<<(count + 255) / 256, 256, 0, st>>>(inst, count, done, stats, params);
  return cudaGetLastError();
}

cudaError_t launch_batch_pending(const BatchInst* inst, int count, int* out, cudaStream_t st) {
  count_launch();
  batch_pending_kernel<<<1, 256, 0, st>>>(inst, count, out);
  return cudaGetLastError();
}

}  // namespace phic
