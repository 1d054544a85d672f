// TMA-staged step kernels for __nv_bfloat16 storage (see step_tma.cuh).
#include "step_tma.cuh"

namespace cm {
template cudaError_t launch_step_tma<__nv_bfloat16>(const void*, const void*, const void*, void*, const void*, const Params&, int*,
                                          int, cudaStream_t);
}  // namespace cm
