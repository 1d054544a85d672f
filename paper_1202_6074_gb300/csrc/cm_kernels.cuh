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
// grids up to this many cells launch the one-cell step with blocks of CM_SMALL_BLOCK threads
#ifndef CM_SMALL_GRID
#define CM_SMALL_GRID 65536
#endif
#ifndef CM_SMALL_BLOCK
#define CM_SMALL_BLOCK 32
#endif
constexpr long long kSmallGrid = CM_SMALL_GRID;
template <class S> constexpr int step_min_blocks() { return sizeof(typename Codec<S>::R) == 8 ? 1 : CM_STEP_MIN_BLOCKS; }
inline dim3 cell_block(int nx) {
    int bx = 32;
    while (bx < kBlock && bx < nx) bx *= 2;
    return dim3(bx, kBlock / bx, 1);
}
// the planes of a step launch: p.z0 .. p.z0 + step_planes(p) - 1
inline int step_planes(const Params& p) { return p.nzc > 0 ? p.nzc : p.nz; }
inline dim3 cell_grid(const Params& p, dim3 b) {
    return dim3((p.nx + b.x - 1) / b.x, (p.ny + b.y - 1) / b.y, step_planes(p));
}

template <class R, bool FIELD = true, bool BIG = false>
__device__ __forceinline__ void load_force(const R* __restrict__ Ff, const PR<R>& p, unsigned cell, R F[3]) {
    if (FIELD && p.has_field) {
        const Ix<BIG> N = cell_count<BIG>(p);
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
    const int z = (int)blockIdx.z + p.z0;
    if (x >= p.nx || y >= p.ny) return;
    using IX = Ix<FT::BIG>;
    const unsigned cell = (unsigned)((z * p.ny + y) * p.nx + x);
    const IX PS = plane_stride<FT::BIG>(p);
    R h[Q];
    gather<D, S, FT::WALLS, FT::BIG, kPullStored>(src, x, y, z, p, h);
    R F[3];
    load_force<R, FT::FIELD, FT::BIG>(Ff, p, cell, F);
    // the collision returns the stored deviations (inverse weights folded into its last sweep)
    collide<D, R, FT, true>(h, F, p, smagorinsky_constant<R, FT::LES>(p, y));
    sfor<Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        Codec<S>::st(dst + (IX(i) * PS + cell), h[slot<D>(i)]);
    });
}

// ---- two cells of a row per thread: k_step_pair in cm_pair.cuh, instantiated per storage in
// inst_pair_*.cu (so that the kernel variants compile in parallel) ----------------------------
template <class S, class FT>
void launch_pair(const void* src, void* dst, const void* Ff, const Params& p, cudaStream_t st);

// ---- density and velocity of the pulled field ----------------------------------------------
template <int D, class S, bool WALLS, bool BIG = false>
__global__ void __launch_bounds__(kBlock) k_moments(const S* __restrict__ src, const typename Codec<S>::R* __restrict__ Ff,
                                                   PR<typename Codec<S>::R> p, double* __restrict__ rho, double* __restrict__ u,
                                                   int z0) {
    using R = typename Codec<S>::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = (int)blockIdx.z + z0;
    if (x >= p.nx || y >= p.ny) return;
    const unsigned cell = (unsigned)((z * p.ny + y) * p.nx + x);
    const Ix<BIG> N = cell_count<BIG>(p);
    R h[Lat<D>::Q];
    gather<D, S, WALLS, BIG>(src, x, y, z, p, h);
    R F[3];
    load_force<R, true, BIG>(Ff, p, cell, F);
    const Hydro<D, R> hy = hydro<D, R>(h, F, p);
    if (rho) rho[cell] = 1.0 + (double)hy.drho;
    if (u) {
        u[cell] = (double)hy.ux;
        u[N + cell] = (double)hy.uy;
        u[2 * N + cell] = (double)hy.uz;
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

// per-block partial sums of {rho, j_x, j_y, j_z, rho |u|^2 / 2} into part[block*5 + k], with the
// momentum j = sum fbar e + F/2 (Eq. velocitycalculation; rho u, or rho0 u in the Sec. 12 form)
template <int D, class S, bool WALLS, bool BIG = false>
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
        gather<D, S, WALLS, BIG>(src, x, y, z, p, h);
        R F[3];
        load_force<R, true, BIG>(Ff, p, (unsigned)c, F);
        const Hydro<D, R> hy = hydro<D, R>(h, F, p);
        const double rho = 1.0 + (double)hy.drho;
        const double ux = (double)hy.ux, uy = (double)hy.uy, uz = (double)hy.uz;
        acc[0] += rho;
        // the momentum j = sum fbar e + F/2 itself (rho u, or rho0 u with reduced compressibility)
        acc[1] += (double)hy.jx;
        acc[2] += (double)hy.jy;
        acc[3] += (double)hy.jz;
        acc[4] += 0.5 * rho * (ux * ux + uy * uy + uz * uz);
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
    if constexpr (FT::UNIT && D == 3) {     // the D3Q27 UNIT variants are pair-kernel variants
        static_assert(sizeof(R) == 4, "D3Q27 UNIT variants are pair-kernel variants");
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
    const dim3 b = p.N <= kSmallGrid ? dim3(CM_SMALL_BLOCK, 1, 1) : cell_block(p.nx), g = cell_grid(p, b);
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
                if constexpr (!F) {
                    // one of the two forms, unforced: its SIMPLE collision with the form fixed at
                    // compile time
                    if (simple_collision(p) && (p.attractor != 0) != (p.reduced != 0)) {
                        if (p.attractor != 0)
                            launch_pair<S, Feat<W, L, false, false, true, false, false, false, true, false>>(src, dst, Ff, p, st);
                        else
                            launch_pair<S, Feat<W, L, false, false, true, false, false, false, false, true>>(src, dst, Ff, p, st);
                        return;
                    }
                }
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
            if constexpr (!F) {
                if (p.F[1] == 0.0 && p.F[2] == 0.0) {      // uniform force along x only
                    launch_step_ft<D, S, Feat<W, L, false, false, false, true, false, true>>(src, dst, Ff, p, st);
                    return;
                }
            }
            launch_step_ft<D, S, Feat<W, L, F, false, false, true>>(src, dst, Ff, p, st);
            return;
        }
    }
    if constexpr (D == 2 && sizeof(R) == 8) {
        // the D2Q9 FP64 step on small grids is bound by the chain of FP64 operations of its
        // collision (GB300's FP64 pipe takes about 64 cycles per warp instruction): with unit
        // higher-order rates the relaxation of orders 3 and 4 drops its products by the rates
        if (p.omega3 == 1.0 && p.omega4 == 1.0) {
            launch_step_ft<D, S, Feat<W, L, F, false, false, true>>(src, dst, Ff, p, st);
            return;
        }
    }
    launch_step_ft<D, S, Feat<W, L, F, false>>(src, dst, Ff, p, st);
}
// The 64-bit-offset step of a D3Q27 grid: for FP32 / 16-bit storage the pair kernel with the
// SIMPLE (unforced, unit higher rates), UNIT (forced, unit higher rates) or general-form
// collision (the general form computes the standard collision too when neither the factorized
// attractor nor reduced compressibility is selected); for FP64 the one-cell kernel with the
// general form.
template <class S, bool W, bool L, bool F>
void launch_step_big_g(const void* src, void* dst, const void* Ff, const Params& p, cudaStream_t st) {
    using R = typename Codec<S>::R;
    if constexpr (sizeof(R) == 4) {
        if (!(p.attractor != 0 || p.reduced)) {
            if constexpr (!F) {
                if (simple_collision(p)) {
                    launch_pair<S, Feat<W, L, false, false, true, false, true>>(src, dst, Ff, p, st);
                    return;
                }
            }
            if (p.omega3 == 1.0 && p.omega4 == 1.0) {
                launch_pair<S, Feat<W, L, F, false, false, true, true>>(src, dst, Ff, p, st);
                return;
            }
        }
        launch_pair<S, Feat<W, L, F, true, false, false, true>>(src, dst, Ff, p, st);
    } else {
        const dim3 b = cell_block(p.nx), g = cell_grid(p, b);
        k_step<3, S, Feat<W, L, F, true, false, false, true>><<<g, b, 0, st>>>((const S*)src, (S*)dst, (const R*)Ff,
                                                                            typed<R>(p));
    }
}
template <class S>
void launch_step_big_impl(const void* src, void* dst, const void* Ff, const Params& p, cudaStream_t st) {
    auto by_field = [&](auto w, auto l) {
        constexpr bool W = decltype(w)::value, L = decltype(l)::value;
        if (p.has_field) launch_step_big_g<S, W, L, true>(src, dst, Ff, p, st);
        else launch_step_big_g<S, W, L, false>(src, dst, Ff, p, st);
    };
    auto by_les = [&](auto w) {
        if (p.les) by_field(w, std::true_type{});
        else by_field(w, std::false_type{});
    };
    if (has_walls(p)) by_les(std::true_type{});
    else by_les(std::false_type{});
}

template <class S>
void launch_step_big(const void* src, void* dst, const void* Ff, const Params& p, cudaStream_t st) {
    launch_step_big_impl<S>(src, dst, Ff, p, st);
}
// instantiated once each, in inst_big_*.cu (so that the variants compile in parallel)
extern template void launch_step_big<double>(const void*, void*, const void*, const Params&, cudaStream_t);
extern template void launch_step_big<float>(const void*, void*, const void*, const Params&, cudaStream_t);
extern template void launch_step_big<__nv_bfloat16>(const void*, void*, const void*, const Params&, cudaStream_t);
extern template void launch_step_big<__half>(const void*, void*, const void*, const Params&, cudaStream_t);

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

// Grids with Q * S >= 2^32 (D3Q27 only): kernel variants with 64-bit element offsets
// (instantiated in inst_big_*.cu): the pair kernel for FP32 / 16-bit storage (p.pair set at
// create), the one-cell kernel for FP64 storage.

template <int D, class S>
cudaError_t launch_step(const void* src, void* dst, const void* Ff, const Params& p, cudaStream_t st) {
    if constexpr (D == 3) {
        if (p.big) {
            launch_step_big<S>(src, dst, Ff, p, st);
            return cudaGetLastError();
        }
    }
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
    if constexpr (D == 3) {
        if (p.big) {
            if (has_walls(p)) k_moments<D, S, true, true><<<g, b, 0, st>>>((const S*)src, (const R*)Ff, typed<R>(p), rho, u, z0);
            else k_moments<D, S, false, true><<<g, b, 0, st>>>((const S*)src, (const R*)Ff, typed<R>(p), rho, u, z0);
            return cudaGetLastError();
        }
    }
    if (has_walls(p)) {
        k_moments<D, S, true><<<g, b, 0, st>>>((const S*)src, (const R*)Ff, typed<R>(p), rho, u, z0);
    } else {
        k_moments<D, S, false><<<g, b, 0, st>>>((const S*)src, (const R*)Ff, typed<R>(p), rho, u, z0);
    }
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
    auto partial = [&](auto walls, auto big) {
        k_reduce_partial<D, S, decltype(walls)::value, decltype(big)::value><<<nb, kRedThreads, 0, st>>>(
            (const S*)src, (const R*)Ff, typed<R>(p), part);
    };
    using T_ = std::true_type;
    using F_ = std::false_type;
    bool big = false;
    if constexpr (D == 3) {
        big = p.big != 0;
        if (big) has_walls(p) ? partial(T_{}, T_{}) : partial(F_{}, T_{});
    }
    if (!big) has_walls(p) ? partial(T_{}, F_{}) : partial(F_{}, F_{});
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
