// Adjoint (reverse mode) of one stream-and-collide step and of the terminal velocity read-out.
//
// Forward step per cell x: g = pull(s_t)(x), s_{t+1}(x) = C(g, F(x)) with C the collision of
// cm_core.cuh. With lambda = dL/ds (post-collision populations, not the encoded deviations):
//   nu(x)       = J_C(g(x))^T lambda_{t+1}(x)             (per-cell vector-Jacobian product)
//   lambda_t    = pull^T nu                               (a permutation: scatter without atomics)
//   dL/dF(x)   += (dC/dF)^T lambda_{t+1}(x)
// The collision is written here in plain central moments of fbar (same function as the
// forward kernel's deviation form):
//   kbar = T(u) g,  post = M(kbar, rho, F),  s = T(u)^-1 post,  u = (sum g e + F/2) / rho.
// Derivatives of the transforms with respect to u use d(T g)_a / du_x = -alpha kbar_(a - e_x)
// (alpha the x exponent of monomial a), so no intermediate sweep state is needed:
//   from the forward transform:  ubar_x -= sum_a kbarbar_a alpha kbar_(a-e_x)
//   from the inverse transform:  ubar_x += sum_a postbar_a alpha post_(a-e_x).
#include "cm_kernels.cuh"
#include "cm_launch.h"

namespace cm {
namespace {

// transpose of the 1D forward transform (f-, f0, f+) -> (m0, m1, m2)
template <class R> __device__ __forceinline__ void fwd1_T(R& a, R& b, R& c, R u) {
    const R m0 = a, m1 = b, m2 = c;
    const R em = R(-1) - u, e0 = -u, ep = R(1) - u;
    a = m0 + em * m1 + em * em * m2;
    b = m0 + e0 * m1 + e0 * e0 * m2;
    c = m0 + ep * m1 + ep * ep * m2;
}
// transpose of the 1D inverse transform (m0, m1, m2) -> (f-, f0, f+), taken through its two
// stages: the shift r1 = u m0 + m1, r2 = u^2 m0 + 2u m1 + m2 (raw moments), then
// f-+ = (r2 -+ r1) / 2, f0 = m0 - r2. Transposed: r1bar = (fp - fm) / 2,
// r2bar = (fm + fp) / 2 - f0, m0bar = f0 + u r1bar + u^2 r2bar, m1bar = r1bar + 2u r2bar,
// m2bar = r2bar.
template <class R> __device__ __forceinline__ void inv1_T(R& a, R& b, R& c, R u, R tu, R uu) {
    const R fm = a, f0 = b, fp = c;
    const R r1 = R(0.5) * (fp - fm);
    const R r2 = fma(R(0.5), fm + fp, -f0);
    a = fma(u, r1, fma(uu, r2, f0));
    b = fma(tu, r2, r1);
    c = r2;
}

template <int D, class R> __device__ __forceinline__ void fwd_T(R (&m)[Lat<D>::Q], R ux, R uy, R uz) {
    constexpr int NL = Lat<D>::Q / 3;
    if constexpr (D == 3) {
#pragma unroll
        for (int t = 0; t < 9; ++t) fwd1_T(m[t], m[9 + t], m[18 + t], uz);
    }
#pragma unroll
    for (int c = 0; c < Lat<D>::NZ; ++c)
#pragma unroll
        for (int a = 0; a < 3; ++a) fwd1_T(m[9 * c + a], m[9 * c + 3 + a], m[9 * c + 6 + a], uy);
#pragma unroll
    for (int l = 0; l < NL; ++l) fwd1_T(m[3 * l], m[3 * l + 1], m[3 * l + 2], ux);
}
template <int D, class R> __device__ __forceinline__ void inv_T(R (&m)[Lat<D>::Q], R ux, R uy, R uz) {
    constexpr int NL = Lat<D>::Q / 3;
    const R tx = ux + ux, ty = uy + uy, tz = uz + uz, qx = ux * ux, qy = uy * uy, qz = uz * uz;
#pragma unroll
    for (int l = 0; l < NL; ++l) inv1_T(m[3 * l], m[3 * l + 1], m[3 * l + 2], ux, tx, qx);
#pragma unroll
    for (int c = 0; c < Lat<D>::NZ; ++c)
#pragma unroll
        for (int a = 0; a < 3; ++a) inv1_T(m[9 * c + a], m[9 * c + 3 + a], m[9 * c + 6 + a], uy, ty, qy);
    if constexpr (D == 3) {
#pragma unroll
        for (int t = 0; t < 9; ++t) inv1_T(m[t], m[9 + t], m[18 + t], uz, tz, qz);
    }
}

// sum_a bar_a * alpha_d(a) * val_(a - e_d) for the three axes
template <int D, class R>
__device__ __forceinline__ void shift_contract(const R (&bar)[Lat<D>::Q], const R (&val)[Lat<D>::Q], R out[3]) {
    constexpr int Q = Lat<D>::Q;
    R s1[3] = {R(0), R(0), R(0)}, s2[3] = {R(0), R(0), R(0)};   // terms with exponent 1 / 2
#pragma unroll
    for (int t = 0; t < Q; ++t) {
        const int a = ex_a(t), b = ex_b(t), c = ex_c(t);
        if (a == 1) s1[0] = fma(bar[t], val[t > 0 ? t - 1 : 0], s1[0]);
        if (a == 2) s2[0] = fma(bar[t], val[t > 0 ? t - 1 : 0], s2[0]);
        if (b == 1) s1[1] = fma(bar[t], val[t > 2 ? t - 3 : 0], s1[1]);
        if (b == 2) s2[1] = fma(bar[t], val[t > 2 ? t - 3 : 0], s2[1]);
        if (c == 1) s1[2] = fma(bar[t], val[t > 8 ? t - 9 : 0], s1[2]);
        if (c == 2) s2[2] = fma(bar[t], val[t > 8 ? t - 9 : 0], s2[2]);
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) out[d] = fma(R(2), s2[d], s1[d]);
}

// Source index of direction i for the pull at (x, y, z): (direction, cell) of the element read.
template <int D, bool WALLS, class R>
__device__ __forceinline__ void pull_source(int i, int x, int y, int z, const PR<R>& p, int& dir, unsigned& cell) {
    int s[3] = {x - Lat<D>::ex(i), y - Lat<D>::ey(i), z - Lat<D>::ez(i)};
    const int n[3] = {p.nx, p.ny, p.nz};
    bool out = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (s[a] < 0 || s[a] >= n[a]) {
            if (!WALLS || p.bc[a] == 0) s[a] += (s[a] < 0) ? n[a] : -n[a];
            else out = true;
        }
    }
    if (out) {
        dir = Lat<D>::opp(i);
        cell = (unsigned)((z * p.ny + y) * p.nx + x);
    } else {
        dir = i;
        cell = (unsigned)((s[2] * p.ny + s[1]) * p.nx + s[0]);
    }
}

// The transpose of the pull (a scatter to the entries the pull of cell (x, y, z) reads): direction
// i of the vector v goes to entry (i, x - e_i) with the periodic wrap, or to (opp(i), x) where the
// link crosses a wall. The per-axis source coordinates and the nine row offsets are computed once,
// as the pull computes them, instead of per direction.
template <int D, bool WALLS, class R>
__device__ __forceinline__ void scatter_pull_T(R* __restrict__ out, int x, int y, int z, const PR<R>& p,
                                               const R (&v)[Lat<D>::Q]) {
    const unsigned N = p.N;
    int xs[3], ys[3], zs[3];
    bool xo[3] = {false, false, false}, yo[3] = {false, false, false}, zo[3] = {false, false, false};
#pragma unroll
    for (int k = 0; k < 3; ++k) {          // slot k <-> e = k - 1, source coordinate = x - e
        int sx = x + 1 - k, sy = y + 1 - k, sz = z + 1 - k;
        if (sx < 0 || sx >= p.nx) {
            if (!WALLS || p.bc[0] != 1) sx += (sx < 0) ? p.nx : -p.nx;
            else xo[k] = true;
        }
        if (sy < 0 || sy >= p.ny) {
            if (!WALLS || p.bc[1] != 1) sy += (sy < 0) ? p.ny : -p.ny;
            else yo[k] = true;
        }
        if constexpr (D == 3) {
            if (sz < 0 || sz >= p.nz) {
                if (!WALLS || p.bc[2] != 1) sz += (sz < 0) ? p.nz : -p.nz;
                else zo[k] = true;
            }
        } else {
            sz = 0;
        }
        xs[k] = sx;
        ys[k] = sy;
        zs[k] = sz;
    }
    const unsigned cell = (unsigned)((z * p.ny + y) * p.nx + x);
    unsigned row[3][3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int b = 0; b < 3; ++b) row[c][b] = (unsigned)((zs[c] * p.ny + ys[b]) * p.nx);
    sfor<Lat<D>::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int a = Lat<D>::ex(i) + 1, b = Lat<D>::ey(i) + 1, c = Lat<D>::ez(i) + 1;
        const unsigned pulled = i * N + row[c][b] + (unsigned)xs[a];
        if constexpr (WALLS) {
            const bool bounced = xo[a] || yo[b] || zo[c];
            out[bounced ? Lat<D>::opp(i) * N + cell : pulled] = v[slot<D>(i)];
        } else {
            out[pulled] = v[slot<D>(i)];
        }
    });
}

template <int D, class S, bool WALLS>
__global__ void __launch_bounds__(kBlock) k_adjoint_terminal(const S* __restrict__ state, const typename Codec<S>::R* __restrict__ Ff,
                                                            PR<typename Codec<S>::R> p, const double* __restrict__ dLdu,
                                                            const double* __restrict__ dLdrho,
                                                            typename Codec<S>::R* __restrict__ lam, double* __restrict__ dLdF) {
    using R = typename Codec<S>::R;
    constexpr int Q = Lat<D>::Q;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= p.nx || y >= p.ny) return;
    const unsigned cell = (unsigned)((z * p.ny + y) * p.nx + x);
    R h[Q];
    gather<D, S, WALLS>(state, x, y, z, p, h);
    R F[3];
    load_force<R>(Ff, p, cell, F);
    const Hydro<D, R> hy = hydro<D, R>(h, F, p);
    const R rho = R(1) + hy.drho, irho = rcp(rho);
    const R mu[3] = {(R)dLdu[cell], (R)dLdu[p.N + cell], D == 3 ? (R)dLdu[2 * p.N + cell] : R(0)};
    const R mr = dLdrho ? (R)dLdrho[cell] : R(0);
    const R u[3] = {hy.ux, hy.uy, hy.uz};
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const R e[3] = {(R)Lat<D>::ex(i), (R)Lat<D>::ey(i), (R)Lat<D>::ez(i)};
        const R nu = mr + irho * (mu[0] * (e[0] - u[0]) + mu[1] * (e[1] - u[1]) + mu[2] * (e[2] - u[2]));
        int dir;
        unsigned sc;
        pull_source<D, WALLS, R>(i, x, y, z, p, dir, sc);
        lam[(unsigned)dir * p.N + sc] = nu;
    }
#pragma unroll
    for (int d = 0; d < D; ++d) dLdF[d * p.N + cell] += (double)(R(0.5) * mu[d] * irho);
}

// 5 resident blocks of 128 threads (at most 102 registers, a 64-byte spill) with the L2
// prefetch below measured fastest at 128^3 and 256^3: 14.0 G cells/s at 256^3 (14.2 with the
// unit-rate variant), against 13.4 with 4 blocks (no spill) and 9.5 with neither the prefetch
// nor the fifth block
#ifndef CM_ADJ_MIN_BLOCKS
#define CM_ADJ_MIN_BLOCKS 5
#endif
#ifndef CM_ADJ_PREFETCH
#define CM_ADJ_PREFETCH 1
#endif
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// How a step's force gradient (dC/dF)^T lambda_{t+1} is accumulated:
//   kAccF64   into the FP64 accumulator dLdF ([3][N] doubles, read and written every step)
//   kAccSeg   into a segment accumulator `seg` in the arithmetic type ([3][N]), which holds the
//             sum over the steps of one checkpoint segment
//   kAccFold  as kAccSeg, then seg (this step's term included) is added into the FP64 dLdF and
//             seg is reset to zero: the last step of a segment in the reverse sweep
// The segment form moves 2 x 12 bytes per cell and step instead of 2 x 24 at FP32 and keeps
// the FP64 accumulation across segments.
enum { kAccF64 = 0, kAccSeg = 1, kAccFold = 2 };

// UNIT: omega_3 = omega_4 = 1 (the default rates), so that the post-collision moments of order
// >= 3 are kappa^M + sigma / 2 and their adjoints need neither rate (fewer live registers)
template <int D, class S, bool WALLS, bool UNIT = false, int ACC = kAccF64>
__global__ void __launch_bounds__(kBlock, CM_ADJ_MIN_BLOCKS) k_adjoint_step(const S* __restrict__ state, const typename Codec<S>::R* __restrict__ Ff,
                                                        PR<typename Codec<S>::R> p, const typename Codec<S>::R* __restrict__ lam_in,
                                                        typename Codec<S>::R* __restrict__ lam_out, double* __restrict__ dLdF,
                                                        typename Codec<S>::R* __restrict__ seg) {
    using R = typename Codec<S>::R;
    constexpr int Q = Lat<D>::Q;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= p.nx || y >= p.ny) return;
    const unsigned cell = (unsigned)((z * p.ny + y) * p.nx + x);
    const size_t NN = p.N;
    const R* __restrict__ lam_c = lam_in + cell;      // lambda_{t+1} of this cell: lam_c[i N]
    double* __restrict__ dF_c = dLdF + cell;
    R* __restrict__ seg_c = seg + cell;
    if (CM_ADJ_PREFETCH) {
        // lambda_{t+1} and the dL/dF accumulator are needed only after the forward
        // recomputation: start bringing them into L2 now so that their loads do not stall
#pragma unroll
        for (int i = 0; i < Q; ++i) prefetch_l2(lam_c + NN * i);
#pragma unroll
        for (int d = 0; d < D; ++d) {
            if constexpr (ACC == kAccF64) prefetch_l2(dF_c + NN * d);
            else prefetch_l2(seg_c + NN * d);
        }
    }

    // ---- forward recomputation (plain central moments of fbar) ----
    R A[Q];                                   // pull (the populations fbar), then kbar
    gather<D, S, WALLS, false, kPullFull>(state, x, y, z, p, A);
    R F[3];
    load_force<R>(Ff, p, cell, F);
    // rho and sum g e: the e = 0 terms are left out (a product by zero is not removed by the
    // compiler: it would change the sign of a zero sum)
    R rho = 0, jx = 0, jy = 0, jz = 0;
    sfor<Q>([&](auto TI) {
        constexpr int t = decltype(TI)::value;
        rho += A[t];
        if constexpr (ex_a(t) == 2) jx += A[t];
        if constexpr (ex_a(t) == 0) jx -= A[t];
        if constexpr (ex_b(t) == 2) jy += A[t];
        if constexpr (ex_b(t) == 0) jy -= A[t];
        if constexpr (D == 3 && ex_c(t) == 2) jz += A[t];
        if constexpr (D == 3 && ex_c(t) == 0) jz -= A[t];
    });
    const R irho = rcp(rho);
    const R u[3] = {(jx + R(0.5) * F[0]) * irho, (jy + R(0.5) * F[1]) * irho, D == 3 ? (jz + R(0.5) * F[2]) * irho : R(0)};
    central_forward<D, R>(A, u[0], u[1], u[2]);      // A = kbar

    const R Fr[3] = {F[0] * irho, F[1] * irho, F[2] * irho};
    const R wnu = rcp(p.tau0);
    const R wb = (p.omega_bulk > R(0)) ? p.omega_bulk : wnu;
    const R w3 = p.omega3, w4 = p.omega4;
    const R third = R(1) / 3;

    // kappa of f (orders >= 2) and post-collision central moments B
    R K[Q];
    R B[Q];
#pragma unroll
    for (int t = 0; t < Q; ++t) K[t] = A[t];
    sfor<2 * D + 1>([&](auto NI) {
        constexpr int n = decltype(NI)::value;
        sfor<Q>([&](auto TI) {
            constexpr int t = decltype(TI)::value;
            if constexpr (n >= 3 && ord(t) == n) {
                constexpr int a = ex_a(t), b = ex_b(t), c = ex_c(t);
                R s = 0;
                if constexpr (a > 0) s += R(a) * Fr[0] * K[t - 1];
                if constexpr (b > 0) s += R(b) * Fr[1] * K[t - 3];
                if constexpr (c > 0) s += R(c) * Fr[2] * K[t - 9];
                K[t] = A[t] + R(0.5) * s;
                constexpr bool even = (a % 2 == 0) && (b % 2 == 0) && (c % 2 == 0);
                constexpr R cM = even ? (R)third_pow((a == 2) + (b == 2) + (c == 2)) : R(0);
                if constexpr (UNIT) {
                    B[t] = cM * rho + R(0.5) * s;
                } else {
                    const R w = (n == 3) ? w3 : w4;
                    B[t] = (R(1) - w) * A[t] + w * cM * rho + (R(1) - R(0.5) * w) * s;
                }
            }
        });
    });
    // order 2: trace with wb, deviator / off-diagonal with wnu
    {
        const int dg[3] = {midx(2, 0, 0), midx(0, 2, 0), midx(0, 0, 2)};
        R P[3] = {0, 0, 0}, tr = 0;
#pragma unroll
        for (int d = 0; d < D; ++d) { P[d] = A[dg[d]] - rho * third; tr += P[d]; }
        const R corr = (wnu - wb) * tr * (R(1) / D);
#pragma unroll
        for (int d = 0; d < D; ++d) B[dg[d]] = rho * third + (R(1) - wnu) * P[d] + corr;
        B[midx(1, 1, 0)] = (R(1) - wnu) * A[midx(1, 1, 0)];
        if constexpr (D == 3) {
            B[midx(1, 0, 1)] = (R(1) - wnu) * A[midx(1, 0, 1)];
            B[midx(0, 1, 1)] = (R(1) - wnu) * A[midx(0, 1, 1)];
        }
    }
    B[0] = A[0];
    B[midx(1, 0, 0)] = A[midx(1, 0, 0)] + F[0];
    B[midx(0, 1, 0)] = A[midx(0, 1, 0)] + F[1];
    if constexpr (D == 3) B[midx(0, 0, 1)] = A[midx(0, 0, 1)] + F[2];

    // ---- reverse ----
    R L[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) L[slot<D>(i)] = __ldg(lam_c + NN * i);
    inv_T<D, R>(L, u[0], u[1], u[2]);           // L = postbar
    R ub[3];
    shift_contract<D, R>(L, B, ub);              // inverse-transform u derivative
    R rb = 0, Fb[3] = {0, 0, 0};

    // first and zeroth order
    Fb[0] += L[midx(1, 0, 0)];
    Fb[1] += L[midx(0, 1, 0)];
    if constexpr (D == 3) Fb[2] += L[midx(0, 0, 1)];

    // orders >= 3, decreasing; B is reused as kappabar accumulators. The source term of moment t
    // along axis d is alpha_d (F_d / rho) kappa_(t - e_d): its derivatives are gathered in
    // G1 / G2 (terms with exponent 1 / 2) as sum kappa_(t - e_d) sbar_t, which give the F and rho
    // adjoints once at the end: Fbar_d += G_d / rho, rhobar -= (F_d / rho) G_d / rho.
#pragma unroll
    for (int t = 0; t < Q; ++t) B[t] = R(0);
    R G1[3] = {R(0), R(0), R(0)}, G2[3] = {R(0), R(0), R(0)};
    const R hw3 = fma(R(-0.5), w3, R(1)), hw4 = fma(R(-0.5), w4, R(1));
    const R om3 = R(1) - w3, om4 = R(1) - w4;
    const R aFr[2][3] = {{Fr[0], Fr[1], Fr[2]}, {Fr[0] + Fr[0], Fr[1] + Fr[1], Fr[2] + Fr[2]}};
    sfor<2 * D + 1>([&](auto NI) {
        constexpr int n = 2 * D - decltype(NI)::value;
        sfor<Q>([&](auto TI) {
            constexpr int t = decltype(TI)::value;
            if constexpr (n >= 3 && ord(t) == n) {
                constexpr int a = ex_a(t), b = ex_b(t), c = ex_c(t);
                constexpr bool even = (a % 2 == 0) && (b % 2 == 0) && (c % 2 == 0);
                const R pb = L[t];
                R sb;
                if constexpr (UNIT) {
                    sb = R(0.5) * (pb + B[t]);
                    if constexpr (even) rb = fma((R)third_pow((a == 2) + (b == 2) + (c == 2)), pb, rb);
                    L[t] = B[t];                                   // kbarbar
                } else {
                    const R w = (n == 3) ? w3 : w4;
                    sb = fma((n == 3) ? hw3 : hw4, pb, R(0.5) * B[t]);
                    if constexpr (even) {
                        constexpr R cM = (R)third_pow((a == 2) + (b == 2) + (c == 2));
                        rb = fma(w * cM, pb, rb);
                    }
                    L[t] = fma((n == 3) ? om3 : om4, pb, B[t]);   // kbarbar
                }
                if constexpr (a == 1) G1[0] = fma(K[t - 1], sb, G1[0]);
                if constexpr (a == 2) G2[0] = fma(K[t - 1], sb, G2[0]);
                if constexpr (a > 0) B[t - 1] = fma(aFr[a - 1][0], sb, B[t - 1]);
                if constexpr (b == 1) G1[1] = fma(K[t - 3], sb, G1[1]);
                if constexpr (b == 2) G2[1] = fma(K[t - 3], sb, G2[1]);
                if constexpr (b > 0) B[t - 3] = fma(aFr[b - 1][1], sb, B[t - 3]);
                if constexpr (c == 1) G1[2] = fma(K[t - 9], sb, G1[2]);
                if constexpr (c == 2) G2[2] = fma(K[t - 9], sb, G2[2]);
                if constexpr (c > 0) B[t - 9] = fma(aFr[c - 1][2], sb, B[t - 9]);
            }
        });
    });
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const R G = fma(R(2), G2[d], G1[d]) * irho;
        Fb[d] += G;
        rb = fma(-Fr[d], G, rb);
    }
    // order 2
    {
        const int dg[3] = {midx(2, 0, 0), midx(0, 2, 0), midx(0, 0, 2)};
        R pb[3] = {0, 0, 0}, trb = 0;
#pragma unroll
        for (int d = 0; d < D; ++d) { pb[d] = L[dg[d]]; trb += pb[d]; }
        const R corr = (wnu - wb) * trb * (R(1) / D);   // R is symmetric
        R sumP = 0;
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const R Pb = (R(1) - wnu) * pb[d] + corr;     // bar of P_d
            L[dg[d]] = Pb + B[dg[d]];
            sumP += Pb;
        }
        rb += third * trb - third * sumP;
        L[midx(1, 1, 0)] = (R(1) - wnu) * L[midx(1, 1, 0)] + B[midx(1, 1, 0)];
        if constexpr (D == 3) {
            L[midx(1, 0, 1)] = (R(1) - wnu) * L[midx(1, 0, 1)] + B[midx(1, 0, 1)];
            L[midx(0, 1, 1)] = (R(1) - wnu) * L[midx(0, 1, 1)] + B[midx(0, 1, 1)];
        }
    }
    // orders 0 and 1: kbarbar = postbar (identity), already in L

    // forward transform: u derivative and transpose
    R ub2[3];
    shift_contract<D, R>(L, A, ub2);
    ub[0] -= ub2[0];
    ub[1] -= ub2[1];
    ub[2] -= ub2[2];
    fwd_T<D, R>(L, u[0], u[1], u[2]);            // L = gbar (slot order)

    // u = (sum g e + F/2) / rho, rho = sum g
    const R ue = -(ub[0] * u[0] + ub[1] * u[1] + ub[2] * u[2]) * irho;
    // L_t += rb + ue + (ub . e_t) / rho, built up axis by axis: X_k = c0 + (k - 1) cx,
    // Y_kj = X_k + (j - 1) cy, then + (l - 1) cz
    {
        const R c0 = rb + ue, cx = ub[0] * irho, cy = ub[1] * irho, cz = ub[2] * irho;
        const R X[3] = {c0 - cx, c0, c0 + cx};
        R Y[9];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            Y[3 + k] = X[k];
            Y[k] = X[k] - cy;
            Y[6 + k] = X[k] + cy;
        }
#pragma unroll
        for (int t = 0; t < Q; ++t) {
            const int l = t / 9;
            const R add = (D == 2 || l == 1) ? Y[t % 9] : (l == 0) ? Y[t % 9] - cz : Y[t % 9] + cz;
            L[t] += add;
        }
    }
    Fb[0] += R(0.5) * irho * ub[0];
    Fb[1] += R(0.5) * irho * ub[1];
    Fb[2] += R(0.5) * irho * ub[2];

    // scatter through the transpose of the pull
    scatter_pull_T<D, WALLS, R>(lam_out, x, y, z, p, L);
#pragma unroll
    for (int d = 0; d < D; ++d) {
        if constexpr (ACC == kAccF64) {
            dF_c[NN * d] += (double)Fb[d];
        } else if constexpr (ACC == kAccSeg) {
            seg_c[NN * d] += Fb[d];
        } else {
            dF_c[NN * d] += (double)(seg_c[NN * d] + Fb[d]);
            seg_c[NN * d] = R(0);
        }
    }
}

}  // namespace

template <int D, class R>
cudaError_t launch_adjoint_terminal(const void* state, const void* Ff, const Params& p, const double* dLdu,
                                    const double* dLdrho, void* lambda, double* dLdF, cudaStream_t st) {
    const dim3 b = cell_block(p.nx), g = cell_grid(p, b);
    if (has_walls(p))
        k_adjoint_terminal<D, R, true><<<g, b, 0, st>>>((const R*)state, (const R*)Ff, typed<R>(p), dLdu, dLdrho, (R*)lambda, dLdF);
    else
        k_adjoint_terminal<D, R, false><<<g, b, 0, st>>>((const R*)state, (const R*)Ff, typed<R>(p), dLdu, dLdrho, (R*)lambda, dLdF);
    return cudaGetLastError();
}

template <int D, class R>
cudaError_t launch_adjoint_step(const void* state, const void* Ff, const Params& p, const void* lam_in, void* lam_out,
                                double* dLdF, void* seg, int acc, cudaStream_t st) {
    const dim3 b = cell_block(p.nx), g = cell_grid(p, b);
    const bool unit = p.omega3 == 1.0 && p.omega4 == 1.0;
    auto go = [&](auto walls, auto u, auto a) {
        k_adjoint_step<D, R, decltype(walls)::value, decltype(u)::value, decltype(a)::value><<<g, b, 0, st>>>(
            (const R*)state, (const R*)Ff, typed<R>(p), (const R*)lam_in, (R*)lam_out, dLdF, (R*)seg);
    };
    auto by_acc = [&](auto walls, auto u) {
        if (acc == kAccSeg) go(walls, u, std::integral_constant<int, kAccSeg>{});
        else if (acc == kAccFold) go(walls, u, std::integral_constant<int, kAccFold>{});
        else go(walls, u, std::integral_constant<int, kAccF64>{});
    };
    using T_ = std::true_type;
    using F_ = std::false_type;
    if (has_walls(p)) unit ? by_acc(T_{}, T_{}) : by_acc(T_{}, F_{});
    else unit ? by_acc(F_{}, T_{}) : by_acc(F_{}, F_{});
    return cudaGetLastError();
}

#define CM_ADJ(D, R)                                                                                               \
    template cudaError_t launch_adjoint_terminal<D, R>(const void*, const void*, const Params&, const double*,     \
                                                       const double*, void*, double*, cudaStream_t);               \
    template cudaError_t launch_adjoint_step<D, R>(const void*, const void*, const Params&, const void*, void*,     \
                                                   double*, void*, int, cudaStream_t);
CM_ADJ(3, double)
CM_ADJ(3, float)
CM_ADJ(2, double)
CM_ADJ(2, float)

}  // namespace cm
