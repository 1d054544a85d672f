// Adjoint kernels (reverse mode of one stream-and-collide step).
#include "cm_kernels.cuh"
#include "cm_launch.h"

namespace cm {
template <int D, class R>
cudaError_t launch_adjoint_terminal(const void*, const void*, const Params&, const double*, const double*, void*,
                                    double*, cudaStream_t) {
    return cudaErrorNotSupported;
}
template <int D, class R>
cudaError_t launch_adjoint_step(const void*, const void*, const Params&, const void*, void*, double*, cudaStream_t) {
    return cudaErrorNotSupported;
}
template cudaError_t launch_adjoint_terminal<3, double>(const void*, const void*, const Params&, const double*, const double*, void*, double*, cudaStream_t);
template cudaError_t launch_adjoint_terminal<3, float>(const void*, const void*, const Params&, const double*, const double*, void*, double*, cudaStream_t);
template cudaError_t launch_adjoint_terminal<2, double>(const void*, const void*, const Params&, const double*, const double*, void*, double*, cudaStream_t);
template cudaError_t launch_adjoint_terminal<2, float>(const void*, const void*, const Params&, const double*, const double*, void*, double*, cudaStream_t);
template cudaError_t launch_adjoint_step<3, double>(const void*, const void*, const Params&, const void*, void*, double*, cudaStream_t);
template cudaError_t launch_adjoint_step<3, float>(const void*, const void*, const Params&, const void*, void*, double*, cudaStream_t);
template cudaError_t launch_adjoint_step<2, double>(const void*, const void*, const Params&, const void*, void*, double*, cudaStream_t);
template cudaError_t launch_adjoint_step<2, float>(const void*, const void*, const Params&, const void*, void*, double*, cudaStream_t);
}  // namespace cm
