// Initial state (paper silent on initialisation): the pre-collision field fbar = f^M - S/2 at
// every cell, stored as the inverse of the pull so that the first step pulls exactly fbar.
#pragma once

#include "cm_core.cuh"

namespace cm {

// ---- equilibrium at the cell -----------------------------------------------------------------
template <int D, class S>
__global__ void __launch_bounds__(kBlock) k_equilibrium(S* __restrict__ dst, const typename Codec<S>::R* __restrict__ Ff,
                                                       PR<typename Codec<S>::R> p, const double* __restrict__ rho,
                                                       const double* __restrict__ u) {
    using R = typename Codec<S>::R;
    constexpr int Q = Lat<D>::Q;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= p.nx || y >= p.ny) return;
    const unsigned cell = (unsigned)((z * p.ny + y) * p.nx + x);
    R F[3];
    load_force<R>(Ff, p, cell, F);
    const double r = rho ? rho[cell] : 1.0;
    double ux = u ? u[cell] : 0.0, uy = u ? u[p.N + cell] : 0.0, uz = (u && D == 3) ? u[2 * p.N + cell] : 0.0;
    if (p.reduced) {   // momentum rho0 u: centre the equilibrium on rho0 u / rho
        ux *= (double)p.rho0 / r;
        uy *= (double)p.rho0 / r;
        uz *= (double)p.rho0 / r;
    }
    R m[Q];
    equilibrium<D, R>(m, (R)r, (R)ux, (R)uy, (R)uz, F);
    sfor<Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr R iw = (R)inv_weight<D>(i);
        Codec<S>::st(dst + ((unsigned)i * p.S + cell), m[slot<D>(i)] * iw);
    });
}

// ---- inverse of the pull -----------------------------------------------------------------------
// s_i(x) = fbar_i(x + e_i), or, when x + e_i is behind a wall, the value whose bounce-back gives
// fbar_{ibar}(x): fbar_{ibar}(x) + 6 w_i (e_i . u_w) in deviation form d (the mean u_w of the
// walls crossed). The three shifted coordinates per axis are formed once, and the 27 (9)
// directions are unrolled at compile time like the pull itself.
// On a slab (bc[2] == 2) the grid's z index also covers the two ghost planes (z = -1 and nz):
// an entry whose x + e_i lies outside the slab's own planes is left unwritten (this slab never
// pulls it; the neighbour holds the same value in its ghost plane), and a reflected entry is
// written only for the slab's own cells (it is pulled by its own cell).
// Offsets are 32-bit unsigned: every offset written or read is in [0, Q*S) even where a ghost
// row's part of it is negative (ghost entries below exist only for e_z = +1, i >= 18).
template <int D, class S>
__global__ void __launch_bounds__(kBlock) k_unstream(const S* __restrict__ fb, S* __restrict__ dst, PR<typename Codec<S>::R> p) {
    using R = typename Codec<S>::R;
    const bool slab = p.bc[2] == 2;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = (int)blockIdx.z - (slab ? 1 : 0);
    if (x >= p.nx || y >= p.ny) return;
    const bool ghost = z < 0 || z >= p.nz;
    int tx[3], ty[3], tz[3];
    bool wx[3] = {false, false, false}, wy[3] = {false, false, false}, wz[3] = {false, false, false};
    bool beyond[3] = {false, false, false};
#pragma unroll
    for (int k = 0; k < 3; ++k) {          // slot k <-> e = k - 1, target coordinate = x + e
        int sx = x + k - 1, sy = y + k - 1, sz = z + k - 1;
        if (sx < 0 || sx >= p.nx) {
            if (p.bc[0] != 1) sx += (sx < 0) ? p.nx : -p.nx;
            else { wx[k] = true; sx = x; }
        }
        if (sy < 0 || sy >= p.ny) {
            if (p.bc[1] != 1) sy += (sy < 0) ? p.ny : -p.ny;
            else { wy[k] = true; sy = y; }
        }
        if (D == 3) {
            if (sz < 0 || sz >= p.nz) {
                if (p.bc[2] == 0) sz += (sz < 0) ? p.nz : -p.nz;
                else if (p.bc[2] == 2) beyond[k] = true;
                else { wz[k] = true; sz = z; }
            }
        } else {
            sz = 0;
        }
        tx[k] = sx;
        ty[k] = sy;
        tz[k] = sz;
    }
    const unsigned cell = (unsigned)((z * p.ny + y) * p.nx + x);
    const unsigned PS = p.S;
    sfor<Lat<D>::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int a = Lat<D>::ex(i) + 1, b = Lat<D>::ey(i) + 1, c = Lat<D>::ez(i) + 1;
        const bool out = wx[a] || wy[b] || wz[c];
        if (out ? ghost : beyond[c]) return;
        R d;
        if (out) {
            // the walls crossed on the way to x + e_i; side 0 below index 0, side 1 above n - 1
            constexpr int sx = (a == 0) ? 0 : 1, sy = (b == 0) ? 0 : 1, sz = (c == 0) ? 0 : 1;
            constexpr R ex = (R)Lat<D>::ex(i), ey = (R)Lat<D>::ey(i), ez = (R)Lat<D>::ez(i);
            R eu = R(0);
            if (wx[a]) eu += ex * p.uw[0][sx][0] + ey * p.uw[0][sx][1] + ez * p.uw[0][sx][2];
            if (wy[b]) eu += ex * p.uw[1][sy][0] + ey * p.uw[1][sy][1] + ez * p.uw[1][sy][2];
            if (wz[c]) eu += ex * p.uw[2][sz][0] + ey * p.uw[2][sz][1] + ez * p.uw[2][sz][2];
            const int cnt = (int)wx[a] + (int)wy[b] + (int)wz[c];
            d = Codec<S>::ld(fb + (Lat<D>::opp(i) * PS + cell)) + R(6) * eu / R(cnt);
        } else {
            const unsigned t = (unsigned)((tz[c] * p.ny + ty[b]) * p.nx + tx[a]);
            d = Codec<S>::ld(fb + (i * PS + t));
        }
        Codec<S>::st(dst + (i * PS + cell), d);
    });
}

template <int D, class S>
cudaError_t launch_init(void* tmp, void* dst, const void* Ff, const Params& p, const double* rho, const double* u,
                        cudaStream_t st) {
    using R = typename Codec<S>::R;
    const dim3 b = cell_block(p.nx), g = cell_grid(p, b);
    k_equilibrium<D, S><<<g, b, 0, st>>>((S*)tmp, (const R*)Ff, typed<R>(p), rho, u);
    dim3 gu = g;
    if (p.bc[2] == 2) gu.z += 2;      // slab: the ghost planes receive the entries leaving the slab
    k_unstream<D, S><<<gu, b, 0, st>>>((const S*)tmp, (S*)dst, typed<R>(p));
    return cudaGetLastError();
}

}  // namespace cm
