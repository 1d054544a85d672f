// Step kernels with 64-bit element offsets (grids with Q * N >= 2^32) for __nv_bfloat16 storage.
#include "cm_pair.cuh"

namespace cm {
template void launch_step_big<__nv_bfloat16>(const void*, void*, const void*, const Params&, cudaStream_t);
}  // namespace cm
