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
__global__ void batch_norm_kernel(const NormItem* items, const NormChunk* chunks, unsigned long long* out) {
  const NormChunk c = chunks[blockIdx.x];
  const NormItem it = items[c.item];
  const int r1 = min(it.n, c.r0 + it.rows_per_chunk);
  double mx = 0.0;
  for (int row = c.r0 + (int)threadIdx.x; row < r1; row += blockDim.x) {
    const int b0 = it.rowptr[row], b1 = it.rowptr[row + 1];
    if (b0 < 0 || b1 < b0 || (long long)b1 > it.nnz) continue;
    double sum = 0.0;
    if (it.f32) {
      const float* v = static_cast<const float*>(it.vals);
      for (int q = b0; q < b1; ++q) sum += fabs((double)v[q]);
    } else {
      const double* v = static_cast<const double*>(it.vals);
      for (int q = b0; q < b1; ++q) sum += fabs(v[q]);
    }
    mx = fmax(mx, sum);
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  __shared__ double wmax[kBlock / 32];
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x / 32); ++w) mx = fmax(mx, wmax[w]);
    atomicMax(out + c.item, (unsigned long long)__double_as_longlong(mx));
  }
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

cudaError_t launch_batch_norms(const NormItem* items, const NormChunk* chunks, int nchunks,
                               unsigned long long* out_bits, cudaStream_t st) {
  if (nchunks < 1) return cudaSuccess;
  count_launch();
  batch_norm_kernel<<<nchunks, kBlock, 0, st>>>(items, chunks, out_bits);
  return cudaGetLastError();
}

}  // namespace phic
