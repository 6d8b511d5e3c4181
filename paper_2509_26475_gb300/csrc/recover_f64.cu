// Recovery kernels of Algorithm 3 in FP64 (see recover_kernels.cuh).
#include "recover_kernels.cuh"

namespace phic {

cudaError_t launch_recover_f64(const SolveArgs& a, cudaStream_t st, int* grid_out) {
  return dispatch_recover<double>(a, st, grid_out);
}
cudaError_t launch_lr_recover_f64(const SolveArgs& a, cudaStream_t st) { return dispatch_lr_recover<double>(a, st); }

}  // namespace phic
