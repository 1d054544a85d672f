// Two-steps-per-pass schedule of the two-cells-per-thread step for float storage (see
// launch_pair_two_steps in cm_pair.cuh).
#include "cm_launch.h"
#include "cm_pair.cuh"

namespace cm {

// feature dispatch as for single steps (launch_step_g / launch_step_l / launch_step_f)
template <bool W, bool L, bool F>
int two_steps_ft(const void* A, void* C, void* ring, const void* Ff, const Params& p, cudaStream_t st) {
    if constexpr (!F) {
        if (simple_collision(p))
            return launch_pair_two_steps<float, Feat<W, L, false, false, true>>(A, C, ring, kTwoStepGroup,
                                                                                 kTwoStepRing, Ff, p, st);
    }
    return launch_pair_two_steps<float, Feat<W, L, F, false>>(A, C, ring, kTwoStepGroup, kTwoStepRing, Ff, p, st);
}
template <bool W, bool L>
int two_steps_l(const void* A, void* C, void* ring, const void* Ff, const Params& p, cudaStream_t st) {
    return p.has_field ? two_steps_ft<W, L, true>(A, C, ring, Ff, p, st) : two_steps_ft<W, L, false>(A, C, ring, Ff, p, st);
}
template <bool W>
int two_steps_w(const void* A, void* C, void* ring, const void* Ff, const Params& p, cudaStream_t st) {
    return p.les ? two_steps_l<W, true>(A, C, ring, Ff, p, st) : two_steps_l<W, false>(A, C, ring, Ff, p, st);
}

int launch_two_steps_f32(const void* A, void* C, void* ring, const void* Ff, const Params& p, cudaStream_t st) {
    if (p.attractor != 0 || p.reduced) return -1;
    const int n = has_walls(p) ? two_steps_w<true>(A, C, ring, Ff, p, st) : two_steps_w<false>(A, C, ring, Ff, p, st);
    return cudaGetLastError() == cudaSuccess ? n : -1;
}

}  // namespace cm
