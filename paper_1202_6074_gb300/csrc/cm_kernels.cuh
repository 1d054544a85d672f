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

// ---- two cells of a row per thread -------------------------------------------------------------
// Cells (x, y, z) and (x + nx/2, y, z) are updated together with the packed FP32 instructions
// (R = F2). They share y and z, hence the y/z wall flags, the row offsets, and the van Driest
// constant; x must be periodic. Each lane is rounded as the scalar FP32 arithmetic rounds it.
#ifndef CM_PAIR_MIN_BLOCKS
#define CM_PAIR_MIN_BLOCKS 4
#endif
template <class S, bool WALLS>
__device__ __forceinline__ void gather_pair(const S* __restrict__ src, int x, int y, int z, const PR<float>& p, F2 (&h)[27]) {
    const unsigned PS = p.S;
    const int half = p.nx >> 1;
    int xa[3], xb[3], ys[3], zs[3];
    bool yo[3] = {false, false, false}, zo[3] = {false, false, false};
#pragma unroll
    for (int k = 0; k < 3; ++k) {          // slot k <-> e = k - 1, source coordinate = x - e
        int sa = x + 1 - k, sb = x + half + 1 - k;     // sa in [-1, half], sb in [half - 1, nx]
        if (sa < 0) sa += p.nx;
        if (sb >= p.nx) sb -= p.nx;
        xa[k] = sa;
        xb[k] = sb;
        int sy = y + 1 - k, sz = z + 1 - k;
        if (sy < 0 || sy >= p.ny) {
            if (!WALLS || p.bc[1] != 1) sy += (sy < 0) ? p.ny : -p.ny;
            else { yo[k] = true; sy = y; }
        }
        if (sz < 0 || sz >= p.nz) {
            if (!WALLS || p.bc[2] != 1) sz += (sz < 0) ? p.wz : -p.wz;
            else { zo[k] = true; sz = z; }
        }
        ys[k] = sy;
        zs[k] = sz;
    }
    const unsigned cellA = (unsigned)((z * p.ny + y) * p.nx + x), cellB = cellA + (unsigned)half;
    unsigned row[3][3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int b = 0; b < 3; ++b) row[c][b] = (unsigned)((zs[c] * p.ny + ys[b]) * p.nx);
    sfor<27>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int a = Lat<3>::ex(i) + 1, b = Lat<3>::ey(i) + 1, c = Lat<3>::ez(i) + 1;
        constexpr float w = (float)weight<3>(i);
        const unsigned base = i * PS + row[c][b];
        if constexpr (WALLS) {
            const bool by = yo[b], bz = zo[c];
            const bool bounced = by || bz;
            const unsigned own = Lat<3>::opp(i) * PS;
            const float da = Codec<S>::ld(src + (bounced ? own + cellA : base + (unsigned)xa[a]));
            const float db = Codec<S>::ld(src + (bounced ? own + cellB : base + (unsigned)xb[a]));
            constexpr int sy = (b == 2) ? 0 : 1, sz = (c == 2) ? 0 : 1;
            float eu = 0.f;
            if constexpr (b != 1) eu += by ? (float(Lat<3>::ex(i)) * p.uw[1][sy][0] + float(Lat<3>::ey(i)) * p.uw[1][sy][1] + float(Lat<3>::ez(i)) * p.uw[1][sy][2]) : 0.f;
            if constexpr (c != 1) eu += bz ? (float(Lat<3>::ex(i)) * p.uw[2][sz][0] + float(Lat<3>::ey(i)) * p.uw[2][sz][1] + float(Lat<3>::ez(i)) * p.uw[2][sz][2]) : 0.f;
            const int cnt = (int)by + (int)bz;
            const float add = 6.f * eu * (cnt == 2 ? 0.5f : 1.f);
            h[slot<3>(i)] = F2(da + add, db + add) * F2(w);
        } else {
            h[slot<3>(i)] = F2(Codec<S>::ld(src + (base + (unsigned)xa[a])), Codec<S>::ld(src + (base + (unsigned)xb[a]))) * F2(w);
        }
    });
}

template <class S, class FT>
__global__ void __launch_bounds__(kBlock, CM_PAIR_MIN_BLOCKS) k_step_pair(const S* __restrict__ src, S* __restrict__ dst,
                                                                          const float* __restrict__ Ff, PR<float> p) {
    const int half = p.nx >> 1;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= half || y >= p.ny) return;
    const unsigned cellA = (unsigned)((z * p.ny + y) * p.nx + x), cellB = cellA + (unsigned)half;
    const unsigned PS = p.S;
    F2 h[27];
    if constexpr (FT::WALLS) {
        const bool near = (p.bc[1] == 1 && (y == 0 || y == p.ny - 1)) || (p.bc[2] == 1 && (z == 0 || z == p.nz - 1));
        if (near) gather_pair<S, true>(src, x, y, z, p, h);
        else gather_pair<S, false>(src, x, y, z, p, h);
    } else {
        gather_pair<S, false>(src, x, y, z, p, h);
    }
    F2 F[3];
    if (FT::FIELD && p.has_field) {
        const unsigned N = p.N;
#pragma unroll
        for (int d = 0; d < 3; ++d) F[d] = F2(__ldg(Ff + (d * N + cellA)), __ldg(Ff + (d * N + cellB)));
    } else {
#pragma unroll
        for (int d = 0; d < 3; ++d) F[d] = F2(p.F[d]);
    }
    collide<3, F2, FT>(h, F, p, smagorinsky_constant<float, FT::LES>(p, y));
    sfor<27>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr float iw = (float)inv_weight<3>(i);
        const F2 v = h[slot<3>(i)] * F2(iw);
        Codec<S>::st(dst + (i * PS + cellA), v.v.x);
        Codec<S>::st(dst + (i * PS + cellB), v.v.y);
    });
}

// ---- density and velocity of the pulled field ----------------------------------------------
template <int D, class S, bool WALLS>
__global__ void __launch_bounds__(kBlock) k_moments(const S* __restrict__ src, const typename Codec<S>::R* __restrict__ Ff,
                                                   PR<typename Codec<S>::R> p, double* __restrict__ rho, double* __restrict__ u) {
    using R = typename Codec<S>::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
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
    if constexpr (D == 3 && sizeof(R) == 4 && !FT::GEN) {
        if (p.pair) {
            const int half = p.nx / 2;
            const dim3 b = cell_block(half);
            const dim3 g((half + b.x - 1) / b.x, (p.ny + b.y - 1) / b.y, p.nz);
            k_step_pair<S, FT><<<g, b, 0, st>>>((const S*)src, (S*)dst, (const float*)Ff, typed<float>(p));
            return;
        }
    }
    const dim3 b = cell_block(p.nx), g = cell_grid(p, b);
    k_step<D, S, FT><<<g, b, 0, st>>>((const S*)src, (S*)dst, (const R*)Ff, typed<R>(p));
}

template <int D, class S, bool W, bool L, bool F>
void launch_step_g(const void* src, void* dst, const void* Ff, const Params& p, cudaStream_t st) {
    if (p.attractor != 0 || p.reduced) launch_step_ft<D, S, Feat<W, L, F, true>>(src, dst, Ff, p, st);
    else launch_step_ft<D, S, Feat<W, L, F, false>>(src, dst, Ff, p, st);
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
cudaError_t launch_moments(const void* src, const void* Ff, const Params& p, double* rho, double* u, cudaStream_t st) {
    using R = typename Codec<S>::R;
    const dim3 b = cell_block(p.nx), g = cell_grid(p, b);
    if (has_walls(p))
        k_moments<D, S, true><<<g, b, 0, st>>>((const S*)src, (const R*)Ff, typed<R>(p), rho, u);
    else
        k_moments<D, S, false><<<g, b, 0, st>>>((const S*)src, (const R*)Ff, typed<R>(p), rho, u);
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
                                                  cudaStream_t);                                           \
    template cudaError_t cm::launch_init<D, S>(void*, void*, const void*, const cm::Params&, const double*,  \
                                               const double*, cudaStream_t);                               \
    template cudaError_t cm::launch_reduce<D, S>(const void*, const void*, const cm::Params&, double*, double*, \
                                                 cudaStream_t);
