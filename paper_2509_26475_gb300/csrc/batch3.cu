// Batched kernel for three resident blocks per SM (up to 85 registers per thread).
#include "batch_kernel.cuh"

namespace phic {

int batch_occupancy_minb3() { return batch_occupancy_of<3>(); }

cudaError_t launch_batch_minb3(const BatchArgs& b, int grid, cudaStream_t st) { return launch_batch_of<3>(b, grid, st); }

}  // namespace phic
