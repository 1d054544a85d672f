// Two-cells-per-thread step kernels of the general collision forms with unit higher-order rates for float storage (see cm_pair.cuh).
#include "cm_pair.cuh"

namespace cm {
CM_PAIR_INSTANTIATE_GEN_UNIT(float)
}  // namespace cm
