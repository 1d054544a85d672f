// D3Q27 stream-and-collide step with TMA staging of the pulled rows in shared memory.
//
// One CTA owns a run of destination rows (TX consecutive cells along x at fixed y, z). For a
// destination row, direction i pulls the source row (y - e_iy, z - e_iz) shifted by -e_ix in x.
// A producer warp streams, for each destination row, the 27 source rows into a ring of shared
// memory stages: the TX-wide row by cp.async.bulk.tensor into a 128-byte aligned slot, and the
// two 16-byte x-halos (the elements just left and right of the row, with the x coordinate
// wrapped around the periodic box) by cp.async.bulk into 16-byte slots, all completing on one
// mbarrier with a transaction count. TX consumer threads wait on the stage, read their 27
// values from shared memory (consecutive x: bank-conflict free), release the stage, then
// collide and store straight to global memory (coalesced rows). Periodic wrap in y and z is
// resolved in the row coordinates; cells whose link crosses a wall take the bounce-back value
// from their own cell in global memory. Every wait is bounded: on expiry the kernel records an
// error code in `err` and returns.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "cm_kernels.cuh"
#include "cm_launch.h"

namespace cm {
namespace {

constexpr unsigned kWaitLimit = 1u << 22;     // try_wait rounds before a wait is declared stuck
constexpr int kMaxTmaDevices = 64;

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait for the completion of the phase with the given parity
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    for (unsigned it = 0; it < kWaitLimit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
// untiled bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned)
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_addr(dst)), "l"((uint64_t)src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1, int c2,
                                            int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, %6}], [%2];"
        ::"r"(smem_addr(dst)), "l"((uint64_t)map), "r"(smem_addr(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
        : "memory");
}

template <class S> __host__ __device__ constexpr int halo() { return 16 / (int)sizeof(S); }   // 16-byte halo
// bytes of one stage: 27 main rows (TX elements each, 128-byte multiples), 27 x 2 halos of 16 B,
// rounded up to 128 so that every stage (and its main rows) starts on a 128-byte boundary
template <class S, int TX> __host__ __device__ constexpr uint32_t stage_bytes() {
    return (uint32_t)(((27 * TX * (int)sizeof(S) + 27 * 2 * 16) + 127) / 128 * 128);
}
template <class S, int TX, int STAGES> __host__ __device__ constexpr size_t tma_smem_bytes() {
    return (size_t)STAGES * stage_bytes<S, TX>() + 2 * STAGES * sizeof(uint64_t) + 128;   // +128: base alignment
}

// HALO = false: the tile spans the whole periodic row (TX == nx), so the x-neighbours of the
// first and last cells are the other end of the same staged row and no halo copies are issued.
template <class S, int TX, int STAGES, class FT, bool HALO>
__global__ void __launch_bounds__(TX + 32, 2) k_step_tma(const __grid_constant__ CUtensorMap map_main,
                                                        const __grid_constant__ CUtensorMap map_halo,
                                                        const S* __restrict__ src, S* __restrict__ dst,
                                                        const typename Codec<S>::R* __restrict__ Ff,
                                                        PR<typename Codec<S>::R> p, int* __restrict__ err) {
    using R = typename Codec<S>::R;
    constexpr int Q = 27;
    constexpr int A = halo<S>();
    constexpr uint32_t kStageBytes = stage_bytes<S, TX>();
    constexpr uint32_t kMainBytes = (uint32_t)(TX * sizeof(S));
    static_assert(kMainBytes % 128 == 0, "main rows must keep 128-byte alignment");
    constexpr uint32_t kTxBytes = (uint32_t)(Q * (TX * sizeof(S) + (HALO ? 2 * 16 : 0)));
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // 128-byte aligned base inside the dynamic shared memory (the allocation has 128 B of slack)
    const uint32_t raw = smem_addr(smem_raw);
    unsigned char* smem = smem_raw + (((raw + 127u) & ~127u) - raw);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * kStageBytes);
    uint64_t* empty = full + STAGES;
    // stage s: main rows at smem + s*kStageBytes + i*kMainBytes; halos after the 27 main rows
    auto main_row = [&](int s, int i) -> S* { return reinterpret_cast<S*>(smem + s * kStageBytes + i * kMainBytes); };
    auto halo_row = [&](int s, int i, int side) -> S* {
        return reinterpret_cast<S*>(smem + s * kStageBytes + Q * kMainBytes + (2 * i + side) * 16);
    };

    const int tid = threadIdx.x;
    const int nxt = p.nx / TX;
    const int nrows = nxt * p.ny * p.nz;           // < 2^31 (cells < 2^31)
    // rows are visited r = blockIdx.x, blockIdx.x + gridDim.x, ...; (xt, y, z) advance with carries
    const int g = (int)gridDim.x;
    const int gx = g % nxt, gy = (g / nxt) % p.ny, gz = g / (nxt * p.ny);
    const int b0 = (int)blockIdx.x;
    const int x00 = b0 % nxt, y00 = (b0 / nxt) % p.ny, z00 = b0 / (nxt * p.ny);
    auto advance = [&](int& xt, int& y, int& z) {
        xt += gx; y += gy; z += gz;
        if (xt >= nxt) { xt -= nxt; ++y; }
        if (y >= p.ny) { y -= p.ny; ++z; }
    };
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], TX / 32);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (tid >= TX) {
        // ---------------- producer warp: lane i issues direction i's three copies ----------------
        const int lane = tid - TX;
        int k = 0;
        int xt = x00, y = y00, z = z00;
        for (int r = b0; r < nrows; r += g, ++k, advance(xt, y, z)) {
            const int s = k % STAGES;
            const uint32_t ph = (uint32_t)(k / STAGES) & 1u;
            bool ok = true;
            if (lane == 0) ok = mbar_wait(&empty[s], ph ^ 1u);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) {
                if (lane == 0) {
                    atomicExch(err, 1);
                    // let the copies already issued land before leaving
                    for (int j = 1; j <= STAGES && k - j >= 0; ++j)
                        mbar_wait(&full[(k - j) % STAGES], (uint32_t)((k - j) / STAGES) & 1u);
                }
                return;
            }
            const int x0 = xt * TX;
            int xl = x0 - A, xr = x0 + TX;
            if (xl < 0) xl = (FT::WALLS && p.bc[0]) ? 0 : xl + p.nx;
            if (xr >= p.nx) xr = (FT::WALLS && p.bc[0]) ? p.nx - A : xr - p.nx;
            if (lane == 0) mbar_arrive_expect_tx(&full[s], kTxBytes);
            __syncwarp();
            if (lane < Q) {
                const int i = lane;
                int ys = y - (i / 3 % 3 - 1), zs = z - (i / 9 - 1);
                if (ys < 0) ys = (FT::WALLS && p.bc[1]) ? 0 : ys + p.ny;
                else if (ys >= p.ny) ys = (FT::WALLS && p.bc[1]) ? p.ny - 1 : ys - p.ny;
                if (zs < 0) zs = (FT::WALLS && p.bc[2]) ? 0 : zs + p.nz;
                else if (zs >= p.nz) zs = (FT::WALLS && p.bc[2]) ? p.nz - 1 : zs - p.nz;
                tma_load_4d(main_row(s, i), &map_main, &full[s], x0, ys, zs, i);
                if constexpr (HALO) {
                    const S* grow = src + ((size_t)i * p.N + ((size_t)zs * p.ny + ys) * p.nx);
                    bulk_load(halo_row(s, i, 0), grow + xl, 16, &full[s]);
                    bulk_load(halo_row(s, i, 1), grow + xr, 16, &full[s]);
                }
            }
        }
        return;
    }

    // ---------------- consumers ----------------
    const unsigned N = p.N;
    const int lane = tid & 31;
    int k = 0;
    int xt = x00, y = y00, z = z00;
    for (int r = b0; r < nrows; r += g, ++k, advance(xt, y, z)) {
        const int s = k % STAGES;
        const uint32_t ph = (uint32_t)(k / STAGES) & 1u;
        if (!mbar_wait(&full[s], ph)) {
            atomicExch(err, 2);
            return;
        }
        const int x = xt * TX + tid;
        const unsigned cell = (unsigned)((z * p.ny + y) * p.nx + x);
        const bool near = FT::WALLS && ((p.bc[0] && (x == 0 || x == p.nx - 1)) || (p.bc[1] && (y == 0 || y == p.ny - 1)) ||
                                        (p.bc[2] && (z == 0 || z == p.nz - 1)));
        R h[Q];
        sfor<Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            constexpr int ex = Lat<3>::ex(i), ey = Lat<3>::ey(i), ez = Lat<3>::ez(i);
            const int j = tid - ex;       // position in the staged row; -1 and TX are the halos
            const S* ptr = main_row(s, i) + j;
            if constexpr (HALO) {
                if constexpr (ex > 0) ptr = (j < 0) ? halo_row(s, i, 0) + (A - 1) : ptr;
                if constexpr (ex < 0) ptr = (j >= TX) ? halo_row(s, i, 1) : ptr;
            } else {          // whole periodic row: wrap inside the staged row
                if constexpr (ex > 0) ptr = (j < 0) ? main_row(s, i) + (TX - 1) : ptr;
                if constexpr (ex < 0) ptr = (j >= TX) ? main_row(s, i) : ptr;
            }
            R d = Codec<S>::ld_shared(ptr);
            if constexpr (FT::WALLS) {
                if (near) {
                    const bool ox = p.bc[0] && (x - ex < 0 || x - ex >= p.nx);
                    const bool oy = p.bc[1] && (y - ey < 0 || y - ey >= p.ny);
                    const bool oz = p.bc[2] && (z - ez < 0 || z - ez >= p.nz);
                    if (ox || oy || oz) {
                        R wx = 0, wy = 0, wz = 0, cnt = 0;
                        if (ox) { const int sd = ex > 0 ? 0 : 1; wx += p.uw[0][sd][0]; wy += p.uw[0][sd][1]; wz += p.uw[0][sd][2]; cnt += 1; }
                        if (oy) { const int sd = ey > 0 ? 0 : 1; wx += p.uw[1][sd][0]; wy += p.uw[1][sd][1]; wz += p.uw[1][sd][2]; cnt += 1; }
                        if (oz) { const int sd = ez > 0 ? 0 : 1; wx += p.uw[2][sd][0]; wy += p.uw[2][sd][1]; wz += p.uw[2][sd][2]; cnt += 1; }
                        d = Codec<S>::ld(src + (Lat<3>::opp(i) * N + cell)) +
                            R(6) * (R(ex) * wx + R(ey) * wy + R(ez) * wz) / cnt;
                    }
                }
            }
            h[slot<3>(i)] = d;
        });
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
        R F[3];
        load_force<R, FT::FIELD>(Ff, p, cell, F);
        collide<3, R, FT>(h, F, p, smagorinsky_constant<R, FT::LES>(p, y));
        sfor<Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            constexpr R iw = (R)inv_weight_scaled<3>(i);
            Codec<S>::st(dst + (i * N + cell), h[slot<3>(i)] * iw);
        });
    }
}

template <class S, int TX, int STAGES, class FT, bool HALO>
cudaError_t launch_tma_ft(const void* map_main, const void* map_halo, const void* src, void* dst, const void* Ff,
                          const Params& p, int* err, int nsm, cudaStream_t st) {
    using R = typename Codec<S>::R;
    constexpr size_t smem = tma_smem_bytes<S, TX, STAGES>();
    // the halos are copied from global memory with 16-byte bulk copies: every row start must be
    // 16-byte aligned (checked here, before anything is launched)
    if (((uintptr_t)src % 16) != 0 || ((size_t)p.nx * sizeof(S)) % 16 != 0 || (p.nx % TX) != 0)
        return cudaErrorMisalignedAddress;
    auto kern = k_step_tma<S, TX, STAGES, FT, HALO>;
    // the shared-memory opt-in is a per-device attribute of the kernel: set it once per device
    static std::atomic<bool> configured[kMaxTmaDevices];
    int dev = 0;
    cudaError_t e0 = cudaGetDevice(&dev);
    if (e0 != cudaSuccess) return e0;
    if (dev < 0 || dev >= kMaxTmaDevices) return cudaErrorInvalidDevice;
    if (!configured[dev].load()) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured[dev].store(true);
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TX + 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const long long nrows = (long long)(p.nx / TX) * p.ny * p.nz;
    long long grid = (long long)per_sm * nsm;
    if (!HALO && (p.nx != TX || p.bc[0])) return cudaErrorInvalidValue;
    if (grid > nrows) grid = nrows;
    kern<<<(unsigned)grid, TX + 32, smem, st>>>(*(const CUtensorMap*)map_main, *(const CUtensorMap*)map_halo,
                                               (const S*)src, (S*)dst, (const R*)Ff, typed<R>(p), err);
    return cudaGetLastError();
}

template <class S, int TX, int STAGES>
cudaError_t launch_tma_tx(const void* mm, const void* mh, const void* src, void* dst, const void* Ff, const Params& p,
                          int* err, int nsm, cudaStream_t st) {
    const bool w = p.bc[0] || p.bc[1] || p.bc[2];
    const bool l = p.les, f = p.has_field;
    const bool halo = !(p.nx == TX && !p.bc[0]);
#define CM_TMA_CASE(W_, L_, F_)                                                                                        \
    if (w == W_ && l == L_ && f == F_)                                                                                 \
        return halo ? launch_tma_ft<S, TX, STAGES, Feat<W_, L_, F_, false>, true>(mm, mh, src, dst, Ff, p, err, nsm, st) \
                    : launch_tma_ft<S, TX, STAGES, Feat<W_, L_, F_, false>, false>(mm, mh, src, dst, Ff, p, err, nsm, st);
    CM_TMA_CASE(false, false, false)
    CM_TMA_CASE(false, false, true)
    CM_TMA_CASE(false, true, false)
    CM_TMA_CASE(false, true, true)
    CM_TMA_CASE(true, false, false)
    CM_TMA_CASE(true, false, true)
    CM_TMA_CASE(true, true, false)
    CM_TMA_CASE(true, true, true)
#undef CM_TMA_CASE
    return cudaErrorInvalidValue;
}

}  // namespace

template <class S>
cudaError_t launch_step_tma(const void* map_main, const void* map_halo, const void* src, void* dst, const void* Ff,
                            const Params& p, int* err, int nsm, cudaStream_t st) {
    const int tx = tma_row_width(p, (int)sizeof(S));
    constexpr int kStages = sizeof(S) == 4 ? 3 : 5;
    if (tx == 256) return launch_tma_tx<S, 256, kStages>(map_main, map_halo, src, dst, Ff, p, err, nsm, st);
    if (tx == 128) return launch_tma_tx<S, 128, kStages>(map_main, map_halo, src, dst, Ff, p, err, nsm, st);
    return cudaErrorInvalidValue;
}

}  // namespace cm
