// Two-cells-per-thread step kernels for __half storage (see cm_pair.cuh).
#include "cm_pair.cuh"

namespace cm {
CM_PAIR_INSTANTIATE(__half)
}  // namespace cm
