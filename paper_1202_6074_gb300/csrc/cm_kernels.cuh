// Kernels and host launch templates, instantiated per (lattice, storage) in inst_*.cu.
#pragma once

#include "cm_core.cuh"

namespace cm {

// Threads per block of the cell kernels and the block shape for a given nx.
constexpr int kBlock = 128;
// Minimum resident blocks per SM requested from the register allocator for the FP32-arithmetic
// step kernel: 8 blocks of 128 threads caps it at 64 registers (measured fastest on GB300 for
// both FP32 and 16-bit storage); FP64 arithmetic is left unconstrained.
#ifndef CM_STEP_MIN_BLOCKS
#define CM_STEP_MIN_BLOCKS 8
#endif
// grids up to this many cells launch the one-cell step with 32-thread blocks
#ifndef CM_SMALL_GRID
#define CM_SMALL_GRID 65536
#endif
constexpr long long kSmallGrid = CM_SMALL_GRID;
template <class S> constexpr int step_min_blocks() { return sizeof(typename Codec<S>::R) == 8 ? 1 : CM_STEP_MIN_BLOCKS; }
inline dim3 cell_block(int nx) {
    int bx = 32;
    while (bx < kBlock && bx < nx) bx *= 2;
    return dim3(bx, kBlock / bx, 1);
}
inline dim3 cell_grid(const Params& p, dim3 b) {
    return dim3((p.nx + b.x - 1) / b.x, (p.ny + b.y - 1) / b.y, p.nz);
}

template <class R, bool FIELD = true>
__device__ __forceinline__ void load_force(const R* __restrict__ Ff, const PR<R>& p, unsigned cell, R F[3]) {
    if (FIELD && p.has_field) {
        const unsigned N = p.N;
        F[0] = __ldg(Ff + cell);
        F[1] = __ldg(Ff + (N + cell));
        F[2] = __ldg(Ff + (2 * N + cell));
    } else {
        F[0] = p.F[0];
        F[1] = p.F[1];
        F[2] = p.F[2];
    }
}

template <class R, bool LES = true>
__device__ __forceinline__ R smagorinsky_constant(const PR<R>& p, int y) {
    if (!LES || !p.les) return R(0);
    R c = p.cs;
    if (p.vd) {
        const R yw = fmin((R)y + R(0.5), (R)p.ny - R(0.5) - (R)y);
        c *= R(1) - exp(-yw * p.vd_utau_nu / p.vd_aplus);
    }
    return c;
}

// ---- fused pull + collide + store --------------------------------------------------------
template <int D, class S, class FT>
__global__ void __launch_bounds__(kBlock, step_min_blocks<S>()) k_step(const S* __restrict__ src, S* __restrict__ dst,
                                                const typename Codec<S>::R* __restrict__ Ff, PR<typename Codec<S>::R> p) {
    using R = typename Codec<S>::R;
    constexpr int Q = Lat<D>::Q;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= p.nx || y >= p.ny) return;
    const unsigned cell = (unsigned)((z * p.ny + y) * p.nx + x);
    const unsigned PS = p.S;
    R h[Q];
    gather<D, S, FT::WALLS>(src, x, y, z, p, h);
    R F[3];
    load_force<R, FT::FIELD>(Ff, p, cell, F);
    collide<D, R, FT>(h, F, p, smagorinsky_constant<R, FT::LES>(p, y));
    sfor<Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr R iw = (R)inv_weight<D>(i);
        Codec<S>::st(dst + (i * PS + cell), h[slot<D>(i)] * iw);
    });
}

// ---- two cells of a row per thread: k_step_pair in cm_pair.cuh, instantiated per storage in
// inst_pair_*.cu (so that the kernel variants compile in parallel) ----------------------------
template <class S, class FT>
void launch_pair(const void* src, void* dst, const void* Ff, const Params& p, cudaStream_t st);

// ---- density and velocity of the pulled field ----------------------------------------------
template <int D, class S, bool WALLS>
__global__ void __launch_bounds__(kBlock) k_moments(const S* __restrict__ src, const typename Codec<S>::R* __restrict__ Ff,
                                                   PR<typename Codec<S>::R> p, double* __restrict__ rho, double* __restrict__ u,
                                                   int z0) {
    using R = typename Codec<S>::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = (int)blockIdx.z + z0;
    if (x >= p.nx || y >= p.ny) return;
    const unsigned cell = (unsigned)((z * p.ny + y) * p.nx + x);
    R h[Lat<D>::Q];
    gather<D, S, WALLS>(src, x, y, z, p, h);
    R F[3];
    load_force<R>(Ff, p, cell, F);
    const Hydro<D, R> hy = hydro<D, R>(h, F, p);
    if (rho) rho[cell] = 1.0 + (double)hy.drho;
    if (u) {
        u[cell] = (double)hy.ux;
        u[p.N + cell] = (double)hy.uy;
        u[2 * p.N + cell] = (double)hy.uz;
    }
}

// ---- deterministic FP64 reductions -------------------------------------------------------
constexpr int kRedThreads = 256;
constexpr int kRedMaxBlocks = 1216;     // 8 blocks on each of 152 SMs

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// per-block partial sums of {rho, rho ux, rho uy, rho uz, rho |u|^2 / 2} into part[block*5 + k]
template <int D, class S, bool WALLS>
__global__ void __launch_bounds__(kRedThreads) k_reduce_partial(const S* __restrict__ src,
                                                               const typename Codec<S>::R* __restrict__ Ff,
                                                               PR<typename Codec<S>::R> p, double* __restrict__ part) {
    using R = typename Codec<S>::R;
    double acc[5] = {0, 0, 0, 0, 0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < p.N; c += stride) {
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
        const double jx = (double)hy.jx, jy = (double)hy.jy, jz = (double)hy.jz;
        const double ux = (double)hy.ux, uy = (double)hy.uy, uz = (double)hy.uz;
        acc[0] += rho;
        acc[1] += rho * ux;
        acc[2] += rho * uy;
        acc[3] += rho * uz;
        acc[4] += 0.5 * rho * (ux * ux + uy * uy + uz * uz);
        (void)jx; (void)jy; (void)jz;
    }
    __shared__ double sh[kRedThreads / 32][5];
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
            double v = (lane < kRedThreads / 32) ? sh[lane][k] : 0.0;
            v = warp_sum(v);
            if (lane == 0) part[blockIdx.x * 5 + k] = v;
        }
    }
}

// sum nblocks partials in a fixed order into out[5]
static __global__ void __launch_bounds__(kRedThreads) k_reduce_final(const double* __restrict__ part, int nblocks,
                                                             double* __restrict__ out) {
    __shared__ double sh[kRedThreads / 32][5];
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
            double v = (lane < kRedThreads / 32) ? sh[lane][k] : 0.0;
            v = warp_sum(v);
            if (lane == 0) out[k] = v;
        }
    }
}

// FP64 [3][N] force field -> arithmetic type
template <class R>
__global__ void k_convert_force(const double* __restrict__ in, R* __restrict__ out, long long n) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) out[k] = (R)in[k];
}

// ------------------------------------------------------------------------------------------
// Host launchers (instantiated in inst_*.cu)
// ------------------------------------------------------------------------------------------
inline bool has_walls(const Params& p) { return p.bc[0] == 1 || p.bc[1] == 1 || p.bc[2] == 1; }

template <int D, class S, class FT>
void launch_step_ft(const void* src, void* dst, const void* Ff, const Params& p, cudaStream_t st) {
    using R = typename Codec<S>::R;
    if constexpr (FT::UNIT) {           // only dispatched to the two-cells-per-thread kernel
        static_assert(D == 3 && sizeof(R) == 4, "UNIT variants are pair-kernel variants");
        launch_pair<S, FT>(src, dst, Ff, p, st);
        return;
    } else if constexpr (D == 3 && sizeof(R) == 4) {
        if (p.pair) {
            launch_pair<S, FT>(src, dst, Ff, p, st);
            return;
        }
    }
    // small grids: one warp per block so that the few blocks spread over as many SMs as possible
    // (the step is latency bound there; 128-thread blocks would leave most SMs idle)
    const dim3 b = p.N <= kSmallGrid ? dim3(32, 1, 1) : cell_block(p.nx), g = cell_grid(p, b);
    k_step<D, S, FT><<<g, b, 0, st>>>((const S*)src, (S*)dst, (const R*)Ff, typed<R>(p));
}

// no force anywhere and unit rates above second order (the SIMPLE variant applies)
inline bool simple_collision(const Params& p) {
    return !p.has_field && p.F[0] == 0.0 && p.F[1] == 0.0 && p.F[2] == 0.0 && p.omega3 == 1.0 && p.omega4 == 1.0;
}

template <int D, class S, bool W, bool L, bool F>
void launch_step_g(const void* src, void* dst, const void* Ff, const Params& p, cudaStream_t st) {
    using R = typename Codec<S>::R;
    if (p.attractor != 0 || p.reduced) {
        if constexpr (D == 3 && sizeof(R) == 4) {
            if (p.pair && p.omega3 == 1.0 && p.omega4 == 1.0) {
                launch_step_ft<D, S, Feat<W, L, F, true, false, true>>(src, dst, Ff, p, st);
                return;
            }
        }
        launch_step_ft<D, S, Feat<W, L, F, true>>(src, dst, Ff, p, st);
        return;
    }
    if constexpr (!F) {
        if (simple_collision(p)) {
            launch_step_ft<D, S, Feat<W, L, false, false, true>>(src, dst, Ff, p, st);
            return;
        }
    }
    if constexpr (D == 3 && sizeof(R) == 4) {
        if (p.pair && p.omega3 == 1.0 && p.omega4 == 1.0) {
            launch_step_ft<D, S, Feat<W, L, F, false, false, true>>(src, dst, Ff, p, st);
            return;
        }
    }
    launch_step_ft<D, S, Feat<W, L, F, false>>(src, dst, Ff, p, st);
}
template <int D, class S, bool W, bool L>
void launch_step_f(const void* src, void* dst, const void* Ff, const Params& p, cudaStream_t st) {
    if (p.has_field) launch_step_g<D, S, W, L, true>(src, dst, Ff, p, st);
    else launch_step_g<D, S, W, L, false>(src, dst, Ff, p, st);
}
template <int D, class S, bool W>
void launch_step_l(const void* src, void* dst, const void* Ff, const Params& p, cudaStream_t st) {
    if (p.les) launch_step_f<D, S, W, true>(src, dst, Ff, p, st);
    else launch_step_f<D, S, W, false>(src, dst, Ff, p, st);
}

template <int D, class S>
cudaError_t launch_step(const void* src, void* dst, const void* Ff, const Params& p, cudaStream_t st) {
    if (has_walls(p)) launch_step_l<D, S, true>(src, dst, Ff, p, st);
    else launch_step_l<D, S, false>(src, dst, Ff, p, st);
    return cudaGetLastError();
}

template <int D, class S>
cudaError_t launch_moments(const void* src, const void* Ff, const Params& p, double* rho, double* u, cudaStream_t st,
                           int z0, int nzc) {
    using R = typename Codec<S>::R;
    const dim3 b = cell_block(p.nx);
    dim3 g = cell_grid(p, b);
    g.z = nzc;
    if (has_walls(p))
        k_moments<D, S, true><<<g, b, 0, st>>>((const S*)src, (const R*)Ff, typed<R>(p), rho, u, z0);
    else
        k_moments<D, S, false><<<g, b, 0, st>>>((const S*)src, (const R*)Ff, typed<R>(p), rho, u, z0);
    return cudaGetLastError();
}

inline int reduce_blocks(const Params& p) {
    long long nb = (p.N + kRedThreads - 1) / kRedThreads;
    return (int)(nb < kRedMaxBlocks ? nb : kRedMaxBlocks);
}

template <int D, class S>
cudaError_t launch_reduce(const void* src, const void* Ff, const Params& p, double* part, double* out, cudaStream_t st) {
    using R = typename Codec<S>::R;
    const int nb = reduce_blocks(p);
    if (has_walls(p))
        k_reduce_partial<D, S, true><<<nb, kRedThreads, 0, st>>>((const S*)src, (const R*)Ff, typed<R>(p), part);
    else
        k_reduce_partial<D, S, false><<<nb, kRedThreads, 0, st>>>((const S*)src, (const R*)Ff, typed<R>(p), part);
    k_reduce_final<<<1, kRedThreads, 0, st>>>(part, nb, out);
    return cudaGetLastError();
}

}  // namespace cm

#include "cm_init.cuh"

// Explicit-instantiation helpers
#define CM_INSTANTIATE(D, S)                                                                               \
    template cudaError_t cm::launch_step<D, S>(const void*, void*, const void*, const cm::Params&, cudaStream_t); \
    template cudaError_t cm::launch_moments<D, S>(const void*, const void*, const cm::Params&, double*, double*, \
                                                  cudaStream_t, int, int);                                 \
    template cudaError_t cm::launch_init<D, S>(void*, const void*, const cm::Params&, const double*,         \
                                               const double*, cudaStream_t, int, int);                     \
    template cudaError_t cm::launch_reduce<D, S>(const void*, const void*, const cm::Params&, double*, double*, \
                                                 cudaStream_t);
