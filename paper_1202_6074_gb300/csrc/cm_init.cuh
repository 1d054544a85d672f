// Initial state (paper silent on initialisation): the pre-collision field fbar = f^M - S/2 at
// every cell, stored as the inverse of the pull so that the first step pulls exactly fbar.
#pragma once

#include "cm_core.cuh"

namespace cm {

// ---- one pass: equilibrium at the cell, written where the first pull reads it --------------
// Each cell x computes its pre-collision field fbar = f^M - S/2 (deviation d = fbar/w - 1) and
// writes direction j where the first pull will read it: s_j(x - e_j) = d_j(x), or, when x - e_j
// is behind a wall, the entry the bounce-back reads, s_jbar(x) = d_j(x) - 6 (e_j . u_w) (u_w
// the mean velocity of the walls crossed; side 0 is below index 0, side 1 above n - 1). Every
// state entry that a pull reads is written by exactly one cell: the cell that pulls it.
// On a slab (bc[2] == 2) the entries pulled across a face land in the ghost planes (z = -1, nz);
// the entries of the own planes that only a neighbour pulls are left unwritten (the neighbour
// holds the same values in its ghost plane). Offsets are 32-bit unsigned: a ghost row below
// has a negative row offset only for e_z = +1 (directions 18..26), so every final offset is
// in [0, Q*S).
template <int D, class S, bool BIG = false>
__global__ void __launch_bounds__(kBlock) k_init(S* __restrict__ dst, const typename Codec<S>::R* __restrict__ Ff,
                                                PR<typename Codec<S>::R> p, const double* __restrict__ rho,
                                                const double* __restrict__ u, int z0) {
    using R = typename Codec<S>::R;
    using IX = Ix<BIG>;
    constexpr int Q = Lat<D>::Q;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = (int)blockIdx.z + z0;
    if (x >= p.nx || y >= p.ny) return;
    const unsigned cell = (unsigned)((z * p.ny + y) * p.nx + x);
    R F[3];
    load_force<R, true, BIG>(Ff, p, cell, F);
    const IX N = cell_count<BIG>(p);
    const double r = rho ? rho[cell] : 1.0;
    double ux = u ? u[cell] : 0.0, uy = u ? u[N + cell] : 0.0, uz = (u && D == 3) ? u[2 * N + cell] : 0.0;
    if (p.reduced) {   // momentum rho0 u: centre the equilibrium on rho0 u / rho
        ux *= (double)p.rho0 / r;
        uy *= (double)p.rho0 / r;
        uz *= (double)p.rho0 / r;
    }
    R m[Q];
    equilibrium<D, R>(m, (R)r, (R)ux, (R)uy, (R)uz, F);

    // target coordinate x - e per axis for slot k <-> e = k - 1, and whether a wall is crossed
    int tx[3], ty[3], tz[3];
    bool wx[3] = {false, false, false}, wy[3] = {false, false, false}, wz[3] = {false, false, false};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        int sx = x + 1 - k, sy = y + 1 - k, sz = z + 1 - k;
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
                else if (p.bc[2] == 1) { wz[k] = true; sz = z; }
                // bc[2] == 2 (slab): the ghost plane at -1 or nz
            }
        } else {
            sz = 0;
        }
        tx[k] = sx;
        ty[k] = sy;
        tz[k] = sz;
    }
    const IX PS = plane_stride<BIG>(p);
    sfor<Q>([&](auto I) {
        constexpr int j = decltype(I)::value;
        constexpr int a = Lat<D>::ex(j) + 1, b = Lat<D>::ey(j) + 1, c = Lat<D>::ez(j) + 1;
        constexpr R iw = (R)inv_weight<D>(j);
        const R d = m[slot<D>(j)] * iw;
        const bool out = wx[a] || wy[b] || wz[c];
        if (out) {
            // the walls crossed going from x to x - e_j: e = +1 crosses the lower wall (side 0)
            constexpr int sx = (a == 2) ? 0 : 1, sy = (b == 2) ? 0 : 1, sz = (c == 2) ? 0 : 1;
            constexpr R ex = (R)Lat<D>::ex(j), ey = (R)Lat<D>::ey(j), ez = (R)Lat<D>::ez(j);
            R eu = R(0);
            if (wx[a]) eu += ex * p.uw[0][sx][0] + ey * p.uw[0][sx][1] + ez * p.uw[0][sx][2];
            if (wy[b]) eu += ex * p.uw[1][sy][0] + ey * p.uw[1][sy][1] + ez * p.uw[1][sy][2];
            if (wz[c]) eu += ex * p.uw[2][sz][0] + ey * p.uw[2][sz][1] + ez * p.uw[2][sz][2];
            const int cnt = (int)wx[a] + (int)wy[b] + (int)wz[c];
            Codec<S>::st(dst + (IX(Lat<D>::opp(j)) * PS + cell), d - R(6) * eu / R(cnt));
        } else {
            const unsigned t = (unsigned)((tz[c] * p.ny + ty[b]) * p.nx + tx[a]);
            Codec<S>::st(dst + (IX(j) * PS + t), d);
        }
    });
}

// the cells of the z-planes z0 .. z0 + nzc - 1 (their writes may land in neighbouring planes:
// every entry has exactly one writer, so chunks of planes may run in any order)
template <int D, class S>
cudaError_t launch_init(void* dst, const void* Ff, const Params& p, const double* rho, const double* u, cudaStream_t st,
                        int z0, int nzc) {
    using R = typename Codec<S>::R;
    const dim3 b = cell_block(p.nx);
    dim3 g = cell_grid(p, b);
    g.z = nzc;
    if constexpr (D == 3) {
        if (p.big) {
            k_init<D, S, true><<<g, b, 0, st>>>((S*)dst, (const R*)Ff, typed<R>(p), rho, u, z0);
            return cudaGetLastError();
        }
    }
    k_init<D, S><<<g, b, 0, st>>>((S*)dst, (const R*)Ff, typed<R>(p), rho, u, z0);
    return cudaGetLastError();
}

}  // namespace cm
