// Step kernel with two cells of a row per thread (packed FP32 arithmetic).
#pragma once

#include "cm_kernels.cuh"

namespace cm {

// Two cells of a row, (x, y, z) and (x + nx/2, y, z) or the adjacent (x0, y, z) and
// (x0 + 1, y, z), are updated together with the packed FP32 instructions (R = F2). They share y
// and z, hence the y/z wall flags, the row offsets, and the van Driest constant; x must be
// periodic. Each lane is rounded as the scalar FP32 arithmetic rounds it.
#ifndef CM_PAIR_MIN_BLOCKS
#define CM_PAIR_MIN_BLOCKS 4
#endif
// Resident blocks per SM the register budget is sized for. The 16-bit steps are bound by
// instruction latency rather than by HBM and gain from more resident warps where the registers
// allow:
//   6 blocks (at most 80 registers) for the unforced SIMPLE collision: +2 % over 5, while 7
//     (72 registers, a 76-byte spill) lose 3 %;
//   6 for the uniform force along x (FX): +1.5 % over 5;
//   5 (at most 96) for the other forced steps without a force field (+5 % on the channel) and
//     for the UNIT collision with a force field (+1.6 % on the isotropic turbulence LES; at 6
//     it would spill over 200 bytes).
// The general relaxation with a force field loses 1 % at 5 blocks and stays at 4 (at most 128
// registers), as do the general forms (they spill twice as much at 5) and all FP32 steps (the
// forced FP32 LES loses 7 % at 5).
#ifndef CM_PAIR_FX_BLOCKS
#define CM_PAIR_FX_BLOCKS (CM_PAIR_MIN_BLOCKS + 2)
#endif
#ifndef CM_PAIR_SIMPLE_BLOCKS
#define CM_PAIR_SIMPLE_BLOCKS (CM_PAIR_MIN_BLOCKS + 2)
#endif
#ifndef CM_PAIR_FIELD_UNIT_BLOCKS
#define CM_PAIR_FIELD_UNIT_BLOCKS (CM_PAIR_MIN_BLOCKS + 1)
#endif
template <class S, class FT>
constexpr int pair_min_blocks() {
    if constexpr (sizeof(S) == 2) {
        if constexpr (FT::FX) return CM_PAIR_FX_BLOCKS;
        if constexpr (FT::FIELD && FT::UNIT && !FT::GEN) return CM_PAIR_FIELD_UNIT_BLOCKS;
        return FT::SIMPLE ? CM_PAIR_SIMPLE_BLOCKS
                          : (!FT::GEN && (!FT::FIELD || FT::UNIT) ? CM_PAIR_MIN_BLOCKS + 1 : CM_PAIR_MIN_BLOCKS);
    }
    return CM_PAIR_MIN_BLOCKS;
}

// Which two cells share a thread: (x, x + nx/2) or the adjacent (x0, x0 + 1), x0 even.
// Adjacent cells read their e_x = 0 populations and write all their populations as one access
// of two entries (e_x = +-1 populations stay two single-entry reads), which removes a third of
// the memory instructions and half of the address arithmetic. Measured on the 256^3 steps:
// +12 % (Taylor-Green) and +14 % (forced LES) at 16-bit storage, +3 % for the forced FP32 LES,
// but -1 % for the unforced FP32 step, which stays on (x, x + nx/2).
template <class S, class FT> constexpr bool pair_adjacent() { return sizeof(S) == 2 || !FT::SIMPLE; }

// Whether the collision returns the stored deviations with the inverse weights folded into its
// last sweep (collide<..., DEV>), or 2^n h, which the store multiplies by 1 / (2^n w) (the
// collision takes the stored deviations either way). The 16-bit steps, which are bound by
// their FP32 arithmetic, fold (the force-field LES BF16 step: +2.2 % at 512^3); the FP32 steps,
// bound by HBM, keep the product at the store.
template <class S, class FT> __host__ __device__ constexpr bool pair_dev() { return sizeof(S) == 2; }

// Blocks of kBlock threads whose x extent divides the pair threads of a row (a multiple of 32:
// nx is a multiple of 64 on this kernel), so that no block is left partly idle at the end of a
// row: 128 x 1 where it divides, else 64 x 2 or 32 x 4 (nx = 384 or 576: 25 % of the threads
// idle with 128-wide blocks).
inline dim3 pair_block(int half) {
    int bx = kBlock;
    while (bx > 32 && half % bx != 0) bx /= 2;
    return dim3(bx, kBlock / bx, 1);
}

// Plane ring of the two-steps-per-pass schedule (launch_pair_two_steps): the intermediate state
// t+1 lives in a small buffer of z-planes instead of a full state buffer. Plane z sits in slot
// z for z < 2 (kept until the end of the pass: the periodic wrap reads them last) and in slot
// 2 + (z - 2) mod slots otherwise; direction planes are `stride` elements apart.
struct Ring {
    unsigned stride;       // elements between direction planes of the ring buffer
    unsigned nxy;          // elements of one z-plane
    int slots;             // ring slots after the two kept planes
    int z0;                // first plane of the launch (blockIdx.z counts from it)
    __device__ __forceinline__ unsigned plane(int z) const {
        return (unsigned)(z < 2 ? z : 2 + (z - 2) % slots) * nxy;
    }
};

// The pair gathers return the stored deviations d (moving-wall term included), not h = w d:
// the collision takes them as they are (see collide).
// RS / RD: the source / destination state is the ring (else a full buffer with stride p.S)
template <class S, bool WALLS, bool RS = false, bool BIG = false>
__device__ __forceinline__ void gather_pair(const S* __restrict__ src, int x, int y, int z, const PR<float>& p, F2 (&h)[27],
                                            const Ring& ring = Ring{}) {
    static_assert(!(RS && BIG), "the plane ring is only used on grids with 32-bit offsets");
    using IX = Ix<BIG>;
    const IX PS = RS ? (IX)ring.stride : plane_stride<BIG>(p);
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
    unsigned cellA, cellB;        // own cells in the source buffer
    unsigned row[3][3];
    if constexpr (RS) {
        cellA = ring.plane(z) + (unsigned)(y * p.nx + x);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const unsigned pl = ring.plane(zs[c]);
#pragma unroll
            for (int b = 0; b < 3; ++b) row[c][b] = pl + (unsigned)(ys[b] * p.nx);
        }
    } else {
        cellA = (unsigned)((z * p.ny + y) * p.nx + x);
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int b = 0; b < 3; ++b) row[c][b] = (unsigned)((zs[c] * p.ny + ys[b]) * p.nx);
    }
    cellB = cellA + (unsigned)half;
    sfor<27>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int a = Lat<3>::ex(i) + 1, b = Lat<3>::ey(i) + 1, c = Lat<3>::ez(i) + 1;
        const IX base = IX(i) * PS + row[c][b];
        if constexpr (WALLS) {
            const bool by = yo[b], bz = zo[c];
            const bool bounced = by || bz;
            const IX own = IX(Lat<3>::opp(i)) * PS;
            float da = Codec<S>::ld(src + (bounced ? own + cellA : base + (unsigned)xa[a]));
            float db = Codec<S>::ld(src + (bounced ? own + cellB : base + (unsigned)xb[a]));
            if (p.moving) {       // half-way bounce-back from a moving wall (see gather_impl)
                constexpr int sy = (b == 2) ? 0 : 1, sz = (c == 2) ? 0 : 1;
                float eu = 0.f;
                if constexpr (b != 1) eu = by ? eu + e_dot<3, i>(p.uw[1][sy]) : eu;
                if constexpr (c != 1) eu = bz ? eu + e_dot<3, i>(p.uw[2][sz]) : eu;
                const float k = wall_factor<float>((int)by + (int)bz);
                da = fmaf(k, eu, da);
                db = fmaf(k, eu, db);
            }
            h[slot<3>(i)] = F2(da, db);
        } else {
            if constexpr (sizeof(S) == 2)   // 64-bit row pointers (measured faster at 16-bit storage)
                h[slot<3>(i)] = F2(Codec<S>::ld(src + xa[a] + base), Codec<S>::ld(src + xb[a] + base));
            else
                h[slot<3>(i)] = F2(Codec<S>::ld(src + (base + (unsigned)xa[a])), Codec<S>::ld(src + (base + (unsigned)xb[a])));
        }
    });
}

// The pull of the adjacent cells (x0, y, z) and (x0 + 1, y, z), x0 even, from a full state
// buffer. Slot k <-> e_x = k - 1 reads columns x - e_x: c0[k] for the first cell, c1[k] for the
// second; the e_x = 0 pair (x0, x0 + 1) is one aligned two-entry read (direction-plane
// strides, row offsets and x0 are even).
template <class S, bool WALLS, bool BIG = false>
__device__ __forceinline__ void gather_adj(const S* __restrict__ src, int x0, int y, int z, const PR<float>& p,
                                           F2 (&h)[27]) {
    using IX = Ix<BIG>;
    const IX PS = plane_stride<BIG>(p);
    const int c0[3] = {x0 + 1, x0, x0 == 0 ? p.nx - 1 : x0 - 1};
    const int c1[3] = {x0 + 2 == p.nx ? 0 : x0 + 2, x0 + 1, x0};
    int ys[3], zs[3];
    bool yo[3] = {false, false, false}, zo[3] = {false, false, false};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
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
    unsigned row[3][3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int b = 0; b < 3; ++b) row[c][b] = (unsigned)((zs[c] * p.ny + ys[b]) * p.nx);
    const unsigned own = (unsigned)((z * p.ny + y) * p.nx + x0);
    sfor<27>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int a = Lat<3>::ex(i) + 1, b = Lat<3>::ey(i) + 1, c = Lat<3>::ez(i) + 1;
        const IX base = IX(i) * PS + row[c][b];
        if constexpr (WALLS) {
            const bool by = yo[b], bz = zo[c];
            const bool bounced = by || bz;
            const IX back = IX(Lat<3>::opp(i)) * PS + own;       // the cells' own reflected entries
            float2 d;
            if constexpr (a == 1) {
                d = Codec<S>::ld2(src + (bounced ? back : base + (unsigned)x0));
            } else {
                d.x = Codec<S>::ld(src + (bounced ? back : base + (unsigned)c0[a]));
                d.y = Codec<S>::ld(src + (bounced ? back + 1u : base + (unsigned)c1[a]));
            }
            if (p.moving) {       // half-way bounce-back from a moving wall (see gather_impl)
                constexpr int sy = (b == 2) ? 0 : 1, sz = (c == 2) ? 0 : 1;
                float eu = 0.f;
                if constexpr (b != 1) eu = by ? eu + e_dot<3, i>(p.uw[1][sy]) : eu;
                if constexpr (c != 1) eu = bz ? eu + e_dot<3, i>(p.uw[2][sz]) : eu;
                const float k = wall_factor<float>((int)by + (int)bz);
                d.x = fmaf(k, eu, d.x);
                d.y = fmaf(k, eu, d.y);
            }
            h[slot<3>(i)] = F2(d.x, d.y);
        } else if constexpr (a == 1) {
            const float2 d = Codec<S>::ld2(src + x0 + base);
            h[slot<3>(i)] = F2(d.x, d.y);
        } else {
            h[slot<3>(i)] = F2(Codec<S>::ld(src + c0[a] + base), Codec<S>::ld(src + c1[a] + base));
        }
    });
}

// gather_adj without walls for a warp none of whose cells pulls across the periodic x edge (its
// columns x0 - 1 .. x0 + 2 all lie in the row): every direction is read through one pointer at
// column x0 of its source row, the e_x = -+1 entries at the constant offsets +1, +2 and -1, 0,
// which the loads take as immediates (the same entries as gather_adj, fewer address operations)
template <class S, bool BIG = false>
__device__ __forceinline__ void gather_adj_inner(const S* __restrict__ src, int x0, int y, int z, const PR<float>& p,
                                                 F2 (&h)[27]) {
    using IX = Ix<BIG>;
    const IX PS = plane_stride<BIG>(p);
    int ys[3], zs[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        int sy = y + 1 - k, sz = z + 1 - k;
        if (sy < 0) sy += p.ny;
        else if (sy >= p.ny) sy -= p.ny;
        if (sz < 0) sz += p.wz;
        else if (sz >= p.nz) sz -= p.wz;
        ys[k] = sy;
        zs[k] = sz;
    }
    const S* __restrict__ px = src + x0;
    sfor<27>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int a = Lat<3>::ex(i) + 1, b = Lat<3>::ey(i) + 1, c = Lat<3>::ez(i) + 1;
        const S* __restrict__ q = px + (IX(i) * PS + (unsigned)((zs[c] * p.ny + ys[b]) * p.nx));
        if constexpr (a == 1) {
            const float2 d = Codec<S>::ld2(q);
            h[slot<3>(i)] = F2(d.x, d.y);
        } else if constexpr (a == 0) {          // e_x = -1: columns x0 + 1, x0 + 2
            h[slot<3>(i)] = F2(Codec<S>::ld(q + 1), Codec<S>::ld(q + 2));
        } else {                                // e_x = +1: columns x0 - 1, x0
            h[slot<3>(i)] = F2(Codec<S>::ld(q - 1), Codec<S>::ld(q));
        }
    });
}

template <class S, class FT, bool RS = false, bool RD = false, bool ADJ = false>
__global__ void __launch_bounds__(kBlock, pair_min_blocks<S, FT>()) k_step_pair(const S* __restrict__ src, S* __restrict__ dst,
                                                                          const float* __restrict__ Ff, PR<float> p,
                                                                          Ring ring) {
    const int half = p.nx >> 1;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = (int)blockIdx.z + ring.z0;     // the ring's group, or the launch's first plane
    if (x >= half || y >= p.ny) return;
    static_assert(!ADJ || (!RS && !RD), "adjacent cells only between full state buffers");
    // global cells (force field) and the destination cells
    const int xa = ADJ ? 2 * x : x;
    const unsigned cellA = (unsigned)((z * p.ny + y) * p.nx + xa), cellB = cellA + (ADJ ? 1u : (unsigned)half);
    const unsigned dA = RD ? ring.plane(z) + (unsigned)(y * p.nx + x) : cellA, dB = dA + (unsigned)half;
    static_assert(!FT::BIG || (!RS && !RD), "the plane ring is only used on grids with 32-bit offsets");
    using IX = Ix<FT::BIG>;
    const IX PS = RD ? (IX)ring.stride : plane_stride<FT::BIG>(p);
    F2 h[27];
    if constexpr (ADJ) {
        // warps are 32 consecutive threads of one row (blockDim.x is a multiple of 32): the warp
        // covers columns 2 x_w .. 2 x_w + 63, and pulls across the periodic x edge only if it holds
        // the row's first or last pair (the test is warp-uniform). The immediate-offset gather of
        // such interior warps measured +1.5 % for the FX channel variant, but -7 % for the 512^3
        // force-field LES and -2.3 % for the unforced Taylor-Green step, which keep gather_adj.
        const int xw = x - (int)(threadIdx.x & 31u);
        const bool inner = FT::FX && xw > 0 && 2 * (xw + 31) + 2 < p.nx;
        bool near = false;
        if constexpr (FT::WALLS)
            near = (p.bc[1] == 1 && (y == 0 || y == p.ny - 1)) || (p.bc[2] == 1 && (z == 0 || z == p.nz - 1));
        if (near) {
            if constexpr (FT::WALLS) gather_adj<S, true, FT::BIG>(src, xa, y, z, p, h);
        } else if (inner) {
            if constexpr (FT::FX) gather_adj_inner<S, FT::BIG>(src, xa, y, z, p, h);
        } else {
            gather_adj<S, false, FT::BIG>(src, xa, y, z, p, h);
        }
    } else if constexpr (FT::WALLS) {
        const bool near = (p.bc[1] == 1 && (y == 0 || y == p.ny - 1)) || (p.bc[2] == 1 && (z == 0 || z == p.nz - 1));
        if (near) gather_pair<S, true, RS, FT::BIG>(src, x, y, z, p, h, ring);
        else gather_pair<S, false, RS, FT::BIG>(src, x, y, z, p, h, ring);
    } else {
        gather_pair<S, false, RS, FT::BIG>(src, x, y, z, p, h, ring);
    }
    F2 F[3];
    if (FT::FIELD && p.has_field) {
        const IX N = cell_count<FT::BIG>(p);
        if constexpr (ADJ) {
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const float2 f = __ldg(reinterpret_cast<const float2*>(Ff + (d * N + cellA)));
                F[d] = F2(f.x, f.y);
            }
        } else {
#pragma unroll
            for (int d = 0; d < 3; ++d) F[d] = F2(__ldg(Ff + (d * N + cellA)), __ldg(Ff + (d * N + cellB)));
        }
    } else {
#pragma unroll
        for (int d = 0; d < 3; ++d) F[d] = F2(p.F[d]);
    }
    constexpr bool DEV = pair_dev<S, FT>();
    collide<3, F2, FT, DEV>(h, F, p, smagorinsky_constant<float, FT::LES>(p, y));
    sfor<27>([&](auto I) {
        constexpr int i = decltype(I)::value;
        const F2 v = DEV ? h[slot<3>(i)] : h[slot<3>(i)] * F2((float)inv_weight_scaled<3>(i));
        if constexpr (ADJ) {
            Codec<S>::st2(dst + dA + (size_t)PS * i, v.v.x, v.v.y);
        } else if constexpr (sizeof(S) == 2) {
            Codec<S>::st(dst + dA + (size_t)PS * i, v.v.x);
            Codec<S>::st(dst + dB + (size_t)PS * i, v.v.y);
        } else {
            Codec<S>::st(dst + (IX(i) * PS + dA), v.v.x);
            Codec<S>::st(dst + (IX(i) * PS + dB), v.v.y);
        }
    });
}

template <class S, class FT>
void launch_pair(const void* src, void* dst, const void* Ff, const Params& p, cudaStream_t st) {
    const int half = p.nx / 2;
    const dim3 b = pair_block(half);
    const dim3 g((half + b.x - 1) / b.x, (p.ny + b.y - 1) / b.y, step_planes(p));
    Ring planes{};
    planes.z0 = p.z0;
    // adjacent cells need both buffers aligned to two entries (buffers passed in by the caller
    // may be offset); the force field is the library's own allocation
    if constexpr (pair_adjacent<S, FT>()) {
        const uintptr_t two = 2 * sizeof(S);
        if ((uintptr_t)src % two == 0 && (uintptr_t)dst % two == 0) {
            k_step_pair<S, FT, false, false, true><<<g, b, 0, st>>>((const S*)src, (S*)dst, (const float*)Ff,
                                                                     typed<float>(p), planes);
            return;
        }
    }
    k_step_pair<S, FT><<<g, b, 0, st>>>((const S*)src, (S*)dst, (const float*)Ff, typed<float>(p), planes);
}

// Two steps per pass (temporal blocking through the L2 cache). Steps t -> t+1 -> t+2 from the
// full buffer A into the full buffer C; the intermediate state t+1 only ever exists in the
// plane ring (see Ring), z-planes in groups of P:
//   for each group [z0, z1):  ring planes z0 .. z1-1 of t+1 from A (reads A planes z0-1 .. z1),
//                             then C planes z0-1 .. z1-2 of t+2 from the ring (reads ring planes
//                             z0-2 .. z1-1, the last P+2 written; group 0 starts at plane 1);
//   at the end:               C planes nz-1 and 0, whose pulls wrap around to ring planes 0, 1
//                             (kept in the first two slots) and nz-2, nz-1.
// Every cell is updated by the same kernel code as in single steps, so the result is bitwise
// the same as two single steps. The ring needs at least P + 2 slots; the recently written ring
// planes are read back while they are still in L2, so each cell's state crosses HBM once per
// two steps (read in A, written in C).
template <class S, class FT>
int launch_pair_two_steps(const void* A, void* C, void* ring, int P, int slots, const void* Ff, const Params& p,
                          cudaStream_t st) {
    const int half = p.nx / 2;
    const dim3 b = cell_block(half);
    const PR<float> q = typed<float>(p);
    const unsigned nxy = (unsigned)p.nx * p.ny;
    Ring rg{(unsigned)(2 + slots) * nxy, nxy, slots, 0};
    auto grid = [&](int planes) { return dim3((half + b.x - 1) / b.x, (p.ny + b.y - 1) / b.y, planes); };
    int launches = 0;
    for (int z0 = 0; z0 < p.nz; z0 += P) {
        const int z1 = z0 + P < p.nz ? z0 + P : p.nz;
        rg.z0 = z0;
        k_step_pair<S, FT, false, true><<<grid(z1 - z0), b, 0, st>>>((const S*)A, (S*)ring, (const float*)Ff, q, rg);
        const int c0 = z0 == 0 ? 1 : z0 - 1, c1 = z1 - 2;
        launches += 1;
        if (c1 >= c0) {
            rg.z0 = c0;
            k_step_pair<S, FT, true, false><<<grid(c1 - c0 + 1), b, 0, st>>>((const S*)ring, (S*)C, (const float*)Ff, q, rg);
            launches += 1;
        }
    }
    for (int z : {p.nz - 1, 0}) {
        rg.z0 = z;
        k_step_pair<S, FT, true, false><<<grid(1), b, 0, st>>>((const S*)ring, (S*)C, (const float*)Ff, q, rg);
        launches += 1;
    }
    return launches;
}

// every feature combination the dispatcher in cm_kernels.cuh can pass
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

// the forced standard collision with unit higher-order rates (the default rates), and its form for
// a uniform force along x (FX)
#define CM_PAIR_INSTANTIATE_UNIT(S)                                                                         \
    template void launch_pair<S, Feat<false, false, false, false, false, true>>(const void*, void*, const void*, const Params&, cudaStream_t); \
    template void launch_pair<S, Feat<false, false, true, false, false, true>>(const void*, void*, const void*, const Params&, cudaStream_t);  \
    template void launch_pair<S, Feat<false, true, false, false, false, true>>(const void*, void*, const void*, const Params&, cudaStream_t);  \
    template void launch_pair<S, Feat<false, true, true, false, false, true>>(const void*, void*, const void*, const Params&, cudaStream_t);   \
    template void launch_pair<S, Feat<true, false, false, false, false, true>>(const void*, void*, const void*, const Params&, cudaStream_t);  \
    template void launch_pair<S, Feat<true, false, true, false, false, true>>(const void*, void*, const void*, const Params&, cudaStream_t);   \
    template void launch_pair<S, Feat<true, true, false, false, false, true>>(const void*, void*, const void*, const Params&, cudaStream_t);   \
    template void launch_pair<S, Feat<true, true, true, false, false, true>>(const void*, void*, const void*, const Params&, cudaStream_t); \
    template void launch_pair<S, Feat<false, false, false, false, false, true, false, true>>(const void*, void*, const void*, const Params&, cudaStream_t); \
    template void launch_pair<S, Feat<false, true, false, false, false, true, false, true>>(const void*, void*, const void*, const Params&, cudaStream_t); \
    template void launch_pair<S, Feat<true, false, false, false, false, true, false, true>>(const void*, void*, const void*, const Params&, cudaStream_t); \
    template void launch_pair<S, Feat<true, true, false, false, false, true, false, true>>(const void*, void*, const void*, const Params&, cudaStream_t);

// the general forms with unit higher-order rates
#define CM_PAIR_INSTANTIATE_GEN_UNIT(S)                                                                     \
    template void launch_pair<S, Feat<false, false, false, true, false, true>>(const void*, void*, const void*, const Params&, cudaStream_t); \
    template void launch_pair<S, Feat<false, false, true, true, false, true>>(const void*, void*, const void*, const Params&, cudaStream_t);  \
    template void launch_pair<S, Feat<false, true, false, true, false, true>>(const void*, void*, const void*, const Params&, cudaStream_t);  \
    template void launch_pair<S, Feat<false, true, true, true, false, true>>(const void*, void*, const void*, const Params&, cudaStream_t);   \
    template void launch_pair<S, Feat<true, false, false, true, false, true>>(const void*, void*, const void*, const Params&, cudaStream_t);  \
    template void launch_pair<S, Feat<true, false, true, true, false, true>>(const void*, void*, const void*, const Params&, cudaStream_t);   \
    template void launch_pair<S, Feat<true, true, false, true, false, true>>(const void*, void*, const void*, const Params&, cudaStream_t);   \
    template void launch_pair<S, Feat<true, true, true, true, false, true>>(const void*, void*, const void*, const Params&, cudaStream_t);

// the unforced SIMPLE collision with the factorized attractor or reduced compressibility fixed at
// compile time
#define CM_PAIR_INSTANTIATE_FORMS(S)                                                                         \
    template void launch_pair<S, Feat<false, false, false, false, true, false, false, false, true, false>>(const void*, void*, const void*, const Params&, cudaStream_t); \
    template void launch_pair<S, Feat<false, true, false, false, true, false, false, false, true, false>>(const void*, void*, const void*, const Params&, cudaStream_t);  \
    template void launch_pair<S, Feat<true, false, false, false, true, false, false, false, true, false>>(const void*, void*, const void*, const Params&, cudaStream_t);  \
    template void launch_pair<S, Feat<true, true, false, false, true, false, false, false, true, false>>(const void*, void*, const void*, const Params&, cudaStream_t);   \
    template void launch_pair<S, Feat<false, false, false, false, true, false, false, false, false, true>>(const void*, void*, const void*, const Params&, cudaStream_t); \
    template void launch_pair<S, Feat<false, true, false, false, true, false, false, false, false, true>>(const void*, void*, const void*, const Params&, cudaStream_t);  \
    template void launch_pair<S, Feat<true, false, false, false, true, false, false, false, false, true>>(const void*, void*, const void*, const Params&, cudaStream_t);  \
    template void launch_pair<S, Feat<true, true, false, false, true, false, false, false, false, true>>(const void*, void*, const void*, const Params&, cudaStream_t);

// the general forms (factorized attractor, reduced compressibility), in translation units of
// their own so that the library builds in parallel
#define CM_PAIR_INSTANTIATE_GEN(S)                                                                          \
    template void launch_pair<S, Feat<false, false, false, true>>(const void*, void*, const void*, const Params&, cudaStream_t); \
    template void launch_pair<S, Feat<false, false, true, true>>(const void*, void*, const void*, const Params&, cudaStream_t);  \
    template void launch_pair<S, Feat<false, true, false, true>>(const void*, void*, const void*, const Params&, cudaStream_t);  \
    template void launch_pair<S, Feat<false, true, true, true>>(const void*, void*, const void*, const Params&, cudaStream_t);   \
    template void launch_pair<S, Feat<true, false, false, true>>(const void*, void*, const void*, const Params&, cudaStream_t);  \
    template void launch_pair<S, Feat<true, false, true, true>>(const void*, void*, const void*, const Params&, cudaStream_t);   \
    template void launch_pair<S, Feat<true, true, false, true>>(const void*, void*, const void*, const Params&, cudaStream_t);   \
    template void launch_pair<S, Feat<true, true, true, true>>(const void*, void*, const void*, const Params&, cudaStream_t);

}  // namespace cm
