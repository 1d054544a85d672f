// Allocation-free variant of the FP64 diagnostics reduction (cmlbm_reduce_noalloc).
//
// Callers such as a host that cannot allocate device memory once set up (a fixed memory
// budget), or a runtime whose memory pool owns the device memory and forbids outside cudaMalloc,
// need the reductions without an allocation. This entry point needs no
// handle and allocates nothing: its per-block partial sums live in the file-scope device array
// `g_reduce_scratch` below (kNoAllocMaxBlocks x 5 doubles = 640 KiB, held by every GPU that
// loads the library until the process exits). Each block of 256 threads covers 1024 cells, so
// the grid, and the scratch it fills, grow with the grid size: at most 16,777,216 cells.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/cmlbm.h"
#include "cm_kernels.cuh"

namespace cm {
namespace {

constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocCellsPerThread = 4;
constexpr int kNoAllocCellsPerBlock = kNoAllocThreads * kNoAllocCellsPerThread;
constexpr int kNoAllocMaxBlocks = 16384;
constexpr long long kNoAllocMaxCells = (long long)kNoAllocMaxBlocks * kNoAllocCellsPerBlock;

// Shared by every call on a device; each call overwrites the partials of the blocks it launches.
static __device__ __align__(256) double g_reduce_scratch[kNoAllocMaxBlocks * 5];

// per-block partial sums over the block's 1024 cells (same per-cell quantities as cmlbm_reduce)
template <int D, class S, bool WALLS>
__global__ void __launch_bounds__(kNoAllocThreads) k_reduce_blocks(const S* __restrict__ src,
                                                                   const typename Codec<S>::R* __restrict__ Ff,
                                                                   PR<typename Codec<S>::R> p, double* __restrict__ part) {
    using R = typename Codec<S>::R;
    double acc[5] = {0, 0, 0, 0, 0};
    const long long base = (long long)blockIdx.x * kNoAllocCellsPerBlock;
#pragma unroll 1
    for (int k = 0; k < kNoAllocCellsPerThread; ++k) {
        const long long c = base + (long long)k * kNoAllocThreads + threadIdx.x;
        if (c >= (long long)p.N) break;
        const int x = (int)(c % p.nx);
        const long long r = c / p.nx;
        const int y = (int)(r % p.ny);
        const int z = (int)(r / p.ny);
        R h[Lat<D>::Q];
        gather<D, S, WALLS>(src, x, y, z, p, h);
        R F[3];
        load_force<R>(Ff, p, (unsigned)c, F);
        const Hydro<D, R> hy = hydro<D, R>(h, F, p);
        const double rho = 1.0 + (double)hy.drho;
        const double ux = (double)hy.ux, uy = (double)hy.uy, uz = (double)hy.uz;
        acc[0] += rho;
        acc[1] += (double)hy.jx;
        acc[2] += (double)hy.jy;
        acc[3] += (double)hy.jz;
        acc[4] += 0.5 * rho * (ux * ux + uy * uy + uz * uz);
    }
    __shared__ double sh[kNoAllocThreads / 32][5];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const double v = warp_sum(acc[k]);
        if (lane == 0) sh[wid][k] = v;
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            double v = (lane < kNoAllocThreads / 32) ? sh[lane][k] : 0.0;
            v = warp_sum(v);
            if (lane == 0) part[blockIdx.x * 5 + k] = v;
        }
    }
}

// sum the nblocks partials in a fixed order into out[5]
__global__ void __launch_bounds__(kNoAllocThreads) k_reduce_blocks_final(const double* __restrict__ part, int nblocks,
                                                                        double* __restrict__ out) {
    __shared__ double sh[kNoAllocThreads / 32][5];
    double acc[5] = {0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < 5; ++k) acc[k] += part[b * 5 + k];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const double v = warp_sum(acc[k]);
        if (lane == 0) sh[wid][k] = v;
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            double v = (lane < kNoAllocThreads / 32) ? sh[lane][k] : 0.0;
            v = warp_sum(v);
            if (lane == 0) out[k] = v;
        }
    }
}

template <int D, class S>
cudaError_t launch_noalloc(const void* state, const void* Ff, const Params& p, double* part, double* out,
                           cudaStream_t st) {
    using R = typename Codec<S>::R;
    const int nb = (int)((p.N + kNoAllocCellsPerBlock - 1) / kNoAllocCellsPerBlock);
    const bool walls = p.bc[0] || p.bc[1] || p.bc[2];
    if (walls)
        k_reduce_blocks<D, S, true><<<nb, kNoAllocThreads, 0, st>>>((const S*)state, (const R*)Ff, typed<R>(p), part);
    else
        k_reduce_blocks<D, S, false><<<nb, kNoAllocThreads, 0, st>>>((const S*)state, (const R*)Ff, typed<R>(p), part);
    k_reduce_blocks_final<<<1, kNoAllocThreads, 0, st>>>(part, nb, out);
    return cudaGetLastError();
}

// Device address of g_reduce_scratch, looked up once per device with that device current and
// kept for the life of the process (a cudaDeviceReset invalidates it; the header says so).
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// The entry point reports failures by status code only (it has no handle to hold a message):
// the message argument documents each check at its call site.
int noalloc_fail(int code, const char* /*why*/) { return code; }

}  // namespace
}  // namespace cm

extern "C" {

int cmlbm_reduce_noalloc(const cmlbm_config* cfg, const void* state, const double uniform_force[3],
                         const void* force_field, double* out) {
    using namespace cm;
    if (!cfg || !state || !out) return noalloc_fail(CMLBM_ERR_INVALID, "cfg, state and out must be non-NULL");
    const cmlbm_config& c = *cfg;
    if (c.lattice != CMLBM_D2Q9 && c.lattice != CMLBM_D3Q27) return noalloc_fail(CMLBM_ERR_INVALID, "unknown lattice");
    if (c.storage < CMLBM_F64 || c.storage > CMLBM_F16) return noalloc_fail(CMLBM_ERR_INVALID, "unknown storage");
    if (c.nx < 1 || c.ny < 1 || c.nz < 1) return noalloc_fail(CMLBM_ERR_INVALID, "grid sizes must be >= 1");
    if (c.lattice == CMLBM_D2Q9 && c.nz != 1) return noalloc_fail(CMLBM_ERR_INVALID, "D2Q9 needs nz == 1");
    for (int a = 0; a < 3; ++a)
        if (c.bc[a] != CMLBM_PERIODIC && c.bc[a] != CMLBM_BOUNCEBACK)
            return noalloc_fail(CMLBM_ERR_INVALID, "bc must be CMLBM_PERIODIC or CMLBM_BOUNCEBACK");
    if (c.reduced_compressibility && !(c.rho0 > 0.0)) return noalloc_fail(CMLBM_ERR_INVALID, "rho0 must be > 0");
    const long long N = (long long)c.nx * c.ny * c.nz;
    if (N > kNoAllocMaxCells)
        return noalloc_fail(CMLBM_ERR_INVALID,
                            "grid too large for the allocation-free reduction: at most 16,777,216 cells");
    if (c.device < 0 || c.device >= kMaxDevices) return noalloc_fail(CMLBM_ERR_INVALID, "device ordinal out of range");

    Params p;
    std::memset(&p, 0, sizeof(p));
    p.nx = c.nx;
    p.ny = c.ny;
    p.nz = c.nz;
    p.N = N;
    p.S = N;
    for (int a = 0; a < 3; ++a) p.bc[a] = c.bc[a];
    std::memcpy(p.uw, c.wall_velocity, sizeof(p.uw));
    for (int d = 0; d < 3; ++d) p.F[d] = uniform_force ? uniform_force[d] : 0.0;
    p.has_field = force_field != nullptr;
    p.reduced = c.reduced_compressibility ? 1 : 0;
    p.rho0 = c.reduced_compressibility ? c.rho0 : 1.0;
    p.tau0 = c.tau;

    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return noalloc_fail(CMLBM_ERR_CUDA, "cudaGetDevice failed");
    if (prev != c.device && cudaSetDevice(c.device) != cudaSuccess)
        return noalloc_fail(CMLBM_ERR_CUDA, "cudaSetDevice failed");
    int rc = CMLBM_OK;
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_scratch_mutex);
        if (!g_scratch_addr[c.device]) {
            void* ptr = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&ptr, g_reduce_scratch);
            if (e != cudaSuccess || !ptr) rc = noalloc_fail(CMLBM_ERR_CUDA, "cudaGetSymbolAddress of the scratch failed");
            else g_scratch_addr[c.device] = ptr;
        }
        scratch = g_scratch_addr[c.device];
    }
    if (rc == CMLBM_OK) {
        cudaStream_t st = (cudaStream_t)c.stream;
        cudaError_t e;
        const bool d3 = c.lattice == CMLBM_D3Q27;
        double* part = (double*)scratch;
        switch (c.storage) {
            case CMLBM_F64: e = d3 ? launch_noalloc<3, double>(state, force_field, p, part, out, st)
                                   : launch_noalloc<2, double>(state, force_field, p, part, out, st); break;
            case CMLBM_F32: e = d3 ? launch_noalloc<3, float>(state, force_field, p, part, out, st)
                                   : launch_noalloc<2, float>(state, force_field, p, part, out, st); break;
            case CMLBM_BF16: e = d3 ? launch_noalloc<3, __nv_bfloat16>(state, force_field, p, part, out, st)
                                    : launch_noalloc<2, __nv_bfloat16>(state, force_field, p, part, out, st); break;
            default: e = d3 ? launch_noalloc<3, __half>(state, force_field, p, part, out, st)
                            : launch_noalloc<2, __half>(state, force_field, p, part, out, st); break;
        }
        if (e != cudaSuccess) rc = noalloc_fail(CMLBM_ERR_CUDA, "reduction kernels failed to launch");
    }
    if (prev >= 0 && prev != c.device) cudaSetDevice(prev);
    return rc;
}

}  // extern "C"
