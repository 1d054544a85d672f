// Two-cells-per-thread step kernels for __nv_bfloat16 storage (see cm_pair.cuh).
#include "cm_pair.cuh"

namespace cm {
CM_PAIR_INSTANTIATE(__nv_bfloat16)
}  // namespace cm
