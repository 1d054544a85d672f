// Two-cells-per-thread step kernels for float storage (see cm_pair.cuh).
#include "cm_pair.cuh"

namespace cm {
CM_PAIR_INSTANTIATE(float)
}  // namespace cm
