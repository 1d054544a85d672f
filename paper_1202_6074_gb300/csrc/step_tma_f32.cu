// TMA-staged step kernels for float storage (see step_tma.cuh).
#include "step_tma.cuh"

namespace cm {
template cudaError_t launch_step_tma<float>(const void*, const void*, const void*, void*, const void*, const Params&, int*,
                                          int, cudaStream_t);
}  // namespace cm
