// Recovery kernels of Algorithm 3 in FP32 (see recover_kernels.cuh).
#include "recover_kernels.cuh"

namespace phic {

cudaError_t launch_recover_f32(const SolveArgs& a, cudaStream_t st, int* grid_out) {
  return dispatch_recover<float>(a, st, grid_out);
}
cudaError_t launch_lr_recover_f32(const SolveArgs& a, cudaStream_t st) { return dispatch_lr_recover<float>(a, st); }

}  // namespace phic
