// Two-cells-per-thread step kernels of the forced collision with unit higher-order rates for __half storage (see cm_pair.cuh).
#include "cm_pair.cuh"

namespace cm {
CM_PAIR_INSTANTIATE_UNIT(__half)
}  // namespace cm
