// Step kernel with two cells of a row per thread (packed FP32 arithmetic).
#pragma once

#include "cm_kernels.cuh"

namespace cm {

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

template <class S, class FT>
void launch_pair(const void* src, void* dst, const void* Ff, const Params& p, cudaStream_t st) {
    const int half = p.nx / 2;
    const dim3 b = cell_block(half);
    const dim3 g((half + b.x - 1) / b.x, (p.ny + b.y - 1) / b.y, p.nz);
    k_step_pair<S, FT><<<g, b, 0, st>>>((const S*)src, (S*)dst, (const float*)Ff, typed<float>(p));
}

// every feature combination the dispatcher in cm_kernels.cuh can pass (the general forms never
// take this kernel)
#define CM_PAIR_INSTANTIATE(S)                                                                              \
    template void launch_pair<S, Feat<false, false, false, false>>(const void*, void*, const void*, const Params&, cudaStream_t); \
    template void launch_pair<S, Feat<false, false, true, false>>(const void*, void*, const void*, const Params&, cudaStream_t);  \
    template void launch_pair<S, Feat<false, true, false, false>>(const void*, void*, const void*, const Params&, cudaStream_t);  \
    template void launch_pair<S, Feat<false, true, true, false>>(const void*, void*, const void*, const Params&, cudaStream_t);   \
    template void launch_pair<S, Feat<true, false, false, false>>(const void*, void*, const void*, const Params&, cudaStream_t);  \
    template void launch_pair<S, Feat<true, false, true, false>>(const void*, void*, const void*, const Params&, cudaStream_t);   \
    template void launch_pair<S, Feat<true, true, false, false>>(const void*, void*, const void*, const Params&, cudaStream_t);   \
    template void launch_pair<S, Feat<true, true, true, false>>(const void*, void*, const void*, const Params&, cudaStream_t);    \
    template void launch_pair<S, Feat<false, false, false, false, true>>(const void*, void*, const void*, const Params&, cudaStream_t); \
    template void launch_pair<S, Feat<false, true, false, false, true>>(const void*, void*, const void*, const Params&, cudaStream_t);  \
    template void launch_pair<S, Feat<true, false, false, false, true>>(const void*, void*, const void*, const Params&, cudaStream_t);  \
    template void launch_pair<S, Feat<true, true, false, false, true>>(const void*, void*, const void*, const Params&, cudaStream_t);

}  // namespace cm
