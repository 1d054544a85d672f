// Two-cells-per-thread step kernels for __half storage: the unforced collision with the factorized
// attractor or reduced compressibility fixed at compile time (see cm_pair.cuh).
#include "cm_pair.cuh"

namespace cm {
CM_PAIR_INSTANTIATE_FORMS(__half)
}  // namespace cm
