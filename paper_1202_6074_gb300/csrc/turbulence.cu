// Turbulence as forcing for the filtered lattice kinetic equation (Sec. 14 of the paper).
//
// The unresolved stresses enter the step as the body force F = rho a', a'_i = -d_j (u'_i u'_j).
// Closure (paper: "any conventional macroscopic turbulence model"): the Smagorinsky model of
// the deviatoric stress, u'_i u'_j - delta_ij u'_k u'_k / 3 = -2 nu_t S_ij, nu_t = C_s^2 |S|,
// |S| = sqrt(2 S:S), lattice spacing 1. Second-order central differences on the periodic box.
// Three passes over the grid:
//   k_hydro_field   rho, u of the current pre-collision field (with the force currently set)
//   k_eddy_stress   T_ij = 2 nu_t S_ij from the velocity differences
//   k_turb_force    F_i = rho sum_j d_j T_ij + (uniform force), written as the handle's force field.
#include "cm_kernels.cuh"
#include "cm_launch.h"

namespace cm {
namespace {

template <int D, class S>
__global__ void __launch_bounds__(kBlock) k_hydro_field(const S* __restrict__ src, const typename Codec<S>::R* __restrict__ Ff,
                                                       PR<typename Codec<S>::R> p, typename Codec<S>::R* __restrict__ q) {
    using R = typename Codec<S>::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= p.nx || y >= p.ny) return;
    const unsigned cell = (unsigned)((z * p.ny + y) * p.nx + x);
    R h[Lat<D>::Q];
    gather<D, S, false>(src, x, y, z, p, h);
    R F[3];
    load_force<R>(Ff, p, cell, F);
    const Hydro<D, R> hy = hydro<D, R>(h, F, p);
    const unsigned N = p.N;
    q[cell] = R(1) + hy.drho;
    q[N + cell] = hy.ux;
    q[2 * N + cell] = hy.uy;
    q[3 * N + cell] = hy.uz;
}

struct Nb {     // periodic neighbour cells along x, y, z (minus, plus)
    unsigned xm, xp, ym, yp, zm, zp;
};
template <class R>
__device__ __forceinline__ Nb neighbours(int x, int y, int z, const PR<R>& p) {
    const int xm = x == 0 ? p.nx - 1 : x - 1, xp = x == p.nx - 1 ? 0 : x + 1;
    const int ym = y == 0 ? p.ny - 1 : y - 1, yp = y == p.ny - 1 ? 0 : y + 1;
    const int zm = z == 0 ? p.nz - 1 : z - 1, zp = z == p.nz - 1 ? 0 : z + 1;
    auto c = [&](int a, int b, int d) { return (unsigned)((d * p.ny + b) * p.nx + a); };
    return {c(xm, y, z), c(xp, y, z), c(x, ym, z), c(x, yp, z), c(x, y, zm), c(x, y, zp)};
}

// T = 2 C^2 |S| S with S_ij = (d_i u_j + d_j u_i) / 2; components xx, yy, zz, xy, xz, yz
template <int D, class R>
__global__ void __launch_bounds__(kBlock) k_eddy_stress(const R* __restrict__ q, PR<R> p, R cs2, R* __restrict__ T) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= p.nx || y >= p.ny) return;
    const unsigned N = p.N;
    const unsigned cell = (unsigned)((z * p.ny + y) * p.nx + x);
    const Nb nb = neighbours<R>(x, y, z, p);
    const R* u = q + N;
    R g[3][3];      // g[i][j] = d_i u_j
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        g[0][j] = R(0.5) * (__ldg(u + j * N + nb.xp) - __ldg(u + j * N + nb.xm));
        g[1][j] = R(0.5) * (__ldg(u + j * N + nb.yp) - __ldg(u + j * N + nb.ym));
        g[2][j] = (D == 3) ? R(0.5) * (__ldg(u + j * N + nb.zp) - __ldg(u + j * N + nb.zm)) : R(0);
    }
    const R sxx = g[0][0], syy = g[1][1], szz = g[2][2];
    const R sxy = R(0.5) * (g[0][1] + g[1][0]), sxz = R(0.5) * (g[0][2] + g[2][0]), syz = R(0.5) * (g[1][2] + g[2][1]);
    const R mag = sqrt(R(2) * (sxx * sxx + syy * syy + szz * szz + R(2) * (sxy * sxy + sxz * sxz + syz * syz)));
    const R k = R(2) * cs2 * mag;
    T[cell] = k * sxx;
    T[N + cell] = k * syy;
    T[2 * N + cell] = k * szz;
    T[3 * N + cell] = k * sxy;
    T[4 * N + cell] = k * sxz;
    T[5 * N + cell] = k * syz;
}

// F_i = rho sum_j (T_ij(x + e_j) - T_ij(x - e_j)) / 2
template <int D, class R>
__global__ void __launch_bounds__(kBlock) k_turb_force(const R* __restrict__ q, const R* __restrict__ T, PR<R> p,
                                                      R* __restrict__ F) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= p.nx || y >= p.ny) return;
    const unsigned N = p.N;
    const unsigned cell = (unsigned)((z * p.ny + y) * p.nx + x);
    const Nb nb = neighbours<R>(x, y, z, p);
    auto t = [&](int comp, unsigned c) { return __ldg(T + comp * N + c); };
    // component index of T_ij: xx 0, yy 1, zz 2, xy 3, xz 4, yz 5
    const R ax = R(0.5) * ((t(0, nb.xp) - t(0, nb.xm)) + (t(3, nb.yp) - t(3, nb.ym)) +
                           (D == 3 ? (t(4, nb.zp) - t(4, nb.zm)) : R(0)));
    const R ay = R(0.5) * ((t(3, nb.xp) - t(3, nb.xm)) + (t(1, nb.yp) - t(1, nb.ym)) +
                           (D == 3 ? (t(5, nb.zp) - t(5, nb.zm)) : R(0)));
    const R az = (D == 3) ? R(0.5) * ((t(4, nb.xp) - t(4, nb.xm)) + (t(5, nb.yp) - t(5, nb.ym)) + (t(2, nb.zp) - t(2, nb.zm)))
                          : R(0);
    const R rho = __ldg(q + cell);
    F[cell] = fma(rho, ax, p.F[0]);          // plus the uniform force set with cmlbm_set_force
    F[N + cell] = fma(rho, ay, p.F[1]);
    F[2 * N + cell] = fma(rho, az, p.F[2]);
}

}  // namespace

template <int D, class S>
cudaError_t launch_turbulence_force(const void* state, void* force, const Params& p, double cs, void* scratch,
                                    cudaStream_t st) {
    using R = typename Codec<S>::R;
    const dim3 b = cell_block(p.nx), g = cell_grid(p, b);
    const PR<R> q = typed<R>(p);
    R* hq = (R*)scratch;                 // [4][N] rho, u
    R* T = hq + 4 * (size_t)p.N;         // [6][N]
    k_hydro_field<D, S><<<g, b, 0, st>>>((const S*)state, (const R*)force, q, hq);
    k_eddy_stress<D, R><<<g, b, 0, st>>>(hq, q, (R)(cs * cs), T);
    k_turb_force<D, R><<<g, b, 0, st>>>(hq, T, q, (R*)force);
    return cudaGetLastError();
}

#define CM_TURB(D, S) \
    template cudaError_t launch_turbulence_force<D, S>(const void*, void*, const Params&, double, void*, cudaStream_t);
CM_TURB(3, double)
CM_TURB(3, float)
CM_TURB(3, __nv_bfloat16)
CM_TURB(3, __half)
CM_TURB(2, double)
CM_TURB(2, float)
CM_TURB(2, __nv_bfloat16)
CM_TURB(2, __half)

}  // namespace cm
