// Step kernels with 64-bit element offsets (grids with Q * N >= 2^32) for double storage.
#include "cm_kernels.cuh"

namespace cm {
template void launch_step_big<double>(const void*, void*, const void*, const Params&, cudaStream_t);
}  // namespace cm
