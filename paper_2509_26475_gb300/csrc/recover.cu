// Single-instance launches of Algorithm 3's recovery phase: dispatch on the storage precision to the
// per-precision units (recover_f32.cu, recover_f64.cu).
#include "kernels.h"

namespace phic {

cudaError_t launch_recover_f32(const SolveArgs& a, cudaStream_t st, int* grid_out);
cudaError_t launch_recover_f64(const SolveArgs& a, cudaStream_t st, int* grid_out);
cudaError_t launch_lr_recover_f32(const SolveArgs& a, cudaStream_t st);
cudaError_t launch_lr_recover_f64(const SolveArgs& a, cudaStream_t st);

cudaError_t launch_lr_recover(const SolveArgs& a, int prec, cudaStream_t st) {
  return prec == PHIC_F32 ? launch_lr_recover_f32(a, st) : launch_lr_recover_f64(a, st);
}

cudaError_t launch_recover(const SolveArgs& a, int prec, cudaStream_t st, int* grid_out) {
  return prec == PHIC_F32 ? launch_recover_f32(a, st, grid_out) : launch_recover_f64(a, st, grid_out);
}

}  // namespace phic
