// Instantiation of the D2Q9 kernels for every storage type, and the force conversion.
#include "cm_kernels.cuh"

CM_INSTANTIATE(2, double)
CM_INSTANTIATE(2, float)
CM_INSTANTIATE(2, __nv_bfloat16)
CM_INSTANTIATE(2, __half)

namespace cm {
cudaError_t launch_convert_force(const double* in, void* out, long long n, bool fp64, cudaStream_t st) {
    const int threads = 256;
    long long blocks = (n + threads - 1) / threads;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    if (fp64)
        k_convert_force<double><<<(int)blocks, threads, 0, st>>>(in, (double*)out, n);
    else
        k_convert_force<float><<<(int)blocks, threads, 0, st>>>(in, (float*)out, n);
    return cudaGetLastError();
}
}  // namespace cm
