// Diagnostics of the C ABI: the FP64 fused multiply-add throughput of the device (the roof that the
// FP64-bound recovery and series kernels are measured against) and a hook that returns Algorithm 1's
// objective coefficients as the selection kernels compute them.
#include <cuda_runtime.h>

#include <cmath>

#include "common.cuh"
#include "phicomb.h"
#include "select_coef.cuh"

namespace phic {
void count_launch();

namespace {

constexpr int kProbeChains = 8;  // independent FMA chains per thread (hide the DFMA latency)
constexpr int kProbeBlocksPerSm = 4;

// Every thread runs kProbeChains independent chains x <- fma(x, a, b), `iters` times each.  a and b are
// launch arguments, so no chain can be folded; the sum is stored only when it equals `never` (never the
// case for the values the host passes), which keeps the chains live without a memory stream.
__global__ void __launch_bounds__(kBlock) fp64_fma_probe_kernel(double* sink, int iters, double a, double b,
                                                                double never) {
  double x[kProbeChains];
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) x[c] = 1e-3 * (double)threadIdx.x + (double)c;
#pragma unroll 4
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) s += x[c];
  if (s == never) sink[0] = s;
}

__global__ void objective_coeffs_kernel(int m, double z, double* out) {
  __shared__ double binom[129];
  if (threadIdx.x == 0) binomial_row(m, binom);
  __syncthreads();
  for (int k = threadIdx.x; k <= m; k += blockDim.x) {
    out[k] = objective_coef(binom[k], z, m - k);
    out[(m + 1) + k] = pow_int(z, m - k);
    out[2 * (m + 1) + k] = binom[k];
  }
}

}  // namespace
}  // namespace phic

using namespace phic;

extern "C" phic_status phic_probe_fp64_fma(int32_t iters, double* sink_dev, int64_t* fmas, phic_stream_t stream) {
  if (iters < 1 || !sink_dev || !fmas) return PHIC_INVALID_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    return PHIC_CUDA_ERROR;
  const int grid = sms * kProbeBlocksPerSm;
  fp64_fma_probe_kernel<<<grid, kBlock, 0, reinterpret_cast<cudaStream_t>(stream)>>>(sink_dev, iters, 0.9999999,
                                                                                      1e-7, -1.0);
  count_launch();
  if (cudaGetLastError() != cudaSuccess) return PHIC_CUDA_ERROR;
  *fmas = (int64_t)grid * kBlock * kProbeChains * (int64_t)iters;
  return PHIC_OK;
}

extern "C" phic_status phic_test_objective_coeffs(int32_t m, double z, double* out_dev, phic_stream_t stream) {
  if (m < 1 || m > 128 || !out_dev || !std::isfinite(z)) return PHIC_INVALID_ARG;
  objective_coeffs_kernel<<<1, 128, 0, reinterpret_cast<cudaStream_t>(stream)>>>(m, z, out_dev);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? PHIC_OK : PHIC_CUDA_ERROR;
}
