// Two-cells-per-thread step kernels of the general collision forms with unit higher-order rates for __nv_bfloat16 storage (see cm_pair.cuh).
#include "cm_pair.cuh"

namespace cm {
CM_PAIR_INSTANTIATE_GEN_UNIT(__nv_bfloat16)
}  // namespace cm
