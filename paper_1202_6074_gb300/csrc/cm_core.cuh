// Device code of the cascaded central-moment step (arXiv:1202.6074) for sm_103a.
//
// Layout: populations are direction-major [Q][N] with N = nx*ny*nz, cell c = (z*ny + y)*nx + x.
// A thread owns one cell and keeps its Q populations in registers in "tensor" order
// t = (ex+1) + 3*(ey+1) + 9*(ez+1); after the forward axis sweeps the same slot holds the
// central moment with exponents (alpha, beta, gamma) = (t%3, t/3%3, t/9).
//
// Arithmetic is carried on deviations from the rest state: h_i = fbar_i - w_i, and central
// moments of h about u. The central moments of the weights about u are the products
// prod_d c_{a_d}(u_d) with c_0 = 1, c_1 = -u, c_2 = 1/3 + u^2, so every quantity the kernel
// rounds is O(u, drho, F) rather than O(1). The algebra is exact: it is the same step as the
// paper's (Secs. 7-11) with the weights' moments moved out analytically.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <type_traits>
#include <utility>

namespace cm {

// Compile-time loop: f(std::integral_constant<int, I>) for I = 0 .. N-1, so that table lookups
// on I (weights, exponents, slots) are constants of the generated code.
template <class F, int... Is>
__host__ __device__ __forceinline__ void sfor_impl(F&& f, std::integer_sequence<int, Is...>) {
    (f(std::integral_constant<int, Is>{}), ...);
}
template <int N, class F> __host__ __device__ __forceinline__ void sfor(F&& f) {
    sfor_impl(f, std::make_integer_sequence<int, N>{});
}

// ------------------------------------------------------------------------------------------
// Parameters (plain data, passed by value to every kernel)
// ------------------------------------------------------------------------------------------
struct Params {
    int nx, ny, nz;
    int bc[3];             // 0 periodic, 1 half-way bounce-back, 2 slab with ghost planes (z only)
    int les;               // Smagorinsky eddy viscosity on
    int vd;                // van Driest damping on (y walls)
    int attractor;         // 0 Maxwellian, 1 factorized
    int reduced;           // reduced compressibility (u = j / rho0)
    int has_field;         // per-cell force field present
    int pair;              // step with two cells of a row per thread (packed FP32, periodic x)
    int big;               // Q * S >= 2^32: kernels with 64-bit element offsets
    int z0, nzc;           // planes z0 .. z0 + nzc - 1 of a step launch (nzc = 0: all planes)
    long long N;           // cells updated (nx ny nz)
    long long S;           // elements between direction planes of a state buffer (N, or nx ny (nz + 2) on a slab)
    double uw[3][2][3];    // wall velocities [axis][side][component]
    double F[3];           // uniform force
    double tau0;           // 1 / omega_nu (base)
    double omega_bulk;     // 0 = follow the effective shear rate
    double omega3, omega4;
    double cs;             // Smagorinsky constant
    double vd_aplus, vd_utau_nu;
    double rho0;
};

// The same parameters in the arithmetic type R (converted once on the host, so kernels do no
// double-precision work on GB300's narrow FP64 path).
template <class R> struct PR {
    int nx, ny, nz;
    int bc[3];
    int les, vd, attractor, reduced, has_field;
    int z0;                // first plane of a step launch (blockIdx.z counts from it)
    unsigned N;            // cells (also the stride of force and moment fields)
    unsigned S;            // direction-plane stride of a state buffer
    unsigned long long N64, S64;   // the same as 64-bit values (kernels with 64-bit offsets)
    int wz;                // z wrap length: nz, or 0 on a slab (the ghost planes are read instead)
    R uw[3][2][3];
    int moving;            // some wall velocity is non-zero (else the pull adds no wall term)
    R F[3];
    R tau0, omega_bulk, omega3, omega4, cs, vd_aplus, vd_utau_nu, rho0;
    R omega_nu;            // 1 / tau0, IEEE-rounded on the host (used by the FP64 collision)
};

template <class R> inline PR<R> typed(const Params& p) {
    PR<R> q;
    q.nx = p.nx; q.ny = p.ny; q.nz = p.nz;
    for (int a = 0; a < 3; ++a) q.bc[a] = p.bc[a];
    q.les = p.les; q.vd = p.vd; q.attractor = p.attractor; q.reduced = p.reduced; q.has_field = p.has_field;
    q.z0 = p.z0;
    q.N = (unsigned)p.N;
    q.S = (unsigned)p.S;
    q.N64 = (unsigned long long)p.N;
    q.S64 = (unsigned long long)p.S;
    q.wz = p.bc[2] == 2 ? 0 : p.nz;
    for (int a = 0; a < 3; ++a)
        for (int s = 0; s < 2; ++s)
            for (int d = 0; d < 3; ++d) q.uw[a][s][d] = (R)p.uw[a][s][d];
    q.moving = 0;
    for (int a = 0; a < 3; ++a)
        for (int s = 0; s < 2; ++s)
            for (int d = 0; d < 3; ++d) q.moving |= p.uw[a][s][d] != 0.0;
    for (int d = 0; d < 3; ++d) q.F[d] = (R)p.F[d];
    q.tau0 = (R)p.tau0; q.omega_bulk = (R)p.omega_bulk; q.omega3 = (R)p.omega3; q.omega4 = (R)p.omega4;
    q.cs = (R)p.cs; q.vd_aplus = (R)p.vd_aplus; q.vd_utau_nu = (R)p.vd_utau_nu; q.rho0 = (R)p.rho0;
    q.omega_nu = (R)(1.0 / p.tau0);
    return q;
}

// Element offsets into state buffers ([Q][S]) and [3][N] fields: 32-bit unsigned while Q * S and
// 3 N stay below 2^32 (checked on the host), else 64-bit (BIG kernel variants). Cell indices
// (z ny + y) nx + x are below 2^31 in both.
template <bool BIG> using Ix = std::conditional_t<BIG, unsigned long long, unsigned>;
template <bool BIG, class P> __host__ __device__ __forceinline__ Ix<BIG> plane_stride(const P& p) {
    if constexpr (BIG) return p.S64;
    else return p.S;
}
template <bool BIG, class P> __host__ __device__ __forceinline__ Ix<BIG> cell_count(const P& p) {
    if constexpr (BIG) return p.N64;
    else return p.N;
}

// reciprocal: IEEE-rounded intrinsic in FP32, plain division in FP64
__device__ __forceinline__ float rcp(float x) { return __frcp_rn(x); }
// the PTX approximations (sqrt.approx.f32, rcp.approx.f32: a single instruction each, within
// a few ulp of the rounded result), used where the eddy viscosity is evaluated (collide)
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }

// Two cells in one value: the packed FP32 instructions of sm_100 and later (FADD2, FMUL2,
// FFMA2) do both lanes in one issue slot, each lane rounded exactly as its scalar FP32
// counterpart. The collision code is written once for R = double, float or F2; products that
// feed a sum are spelled out as fma() so that the packed form keeps the fused rounding.
struct F2 {
    float2 v;
    F2() = default;
    __device__ __forceinline__ F2(float s) : v(make_float2(s, s)) {}
    __device__ __forceinline__ F2(float a, float b) : v(make_float2(a, b)) {}
};
__device__ __forceinline__ F2 f2(float2 x) {
    F2 r;
    r.v = x;
    return r;
}
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return f2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator-(F2 a) { return F2(-a.v.x, -a.v.y); }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return f2(__fadd2_rn(a.v, make_float2(-b.v.x, -b.v.y))); }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return f2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ F2& operator+=(F2& a, F2 b) { return a = a + b; }
__device__ __forceinline__ F2& operator*=(F2& a, F2 b) { return a = a * b; }
// (declaring fma/sqrt for F2 in this namespace hides the global ones: restate the scalar forms)
__device__ __forceinline__ float fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma(double a, double b, double c) { return ::fma(a, b, c); }
__device__ __forceinline__ float sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double sqrt(double x) { return ::sqrt(x); }
__device__ __forceinline__ F2 fma(F2 a, F2 b, F2 c) { return f2(__ffma2_rn(a.v, b.v, c.v)); }
__device__ __forceinline__ F2 rcp(F2 x) { return F2(__frcp_rn(x.v.x), __frcp_rn(x.v.y)); }
__device__ __forceinline__ F2 sqrt(F2 x) { return F2(sqrtf(x.v.x), sqrtf(x.v.y)); }
// square root and reciprocal of the eddy-viscosity relaxation time: the approximations in FP32
// (measured +4 % on the 16-bit wall-bounded LES step, which is bound by its FP32 arithmetic),
// the rounded operations in FP64
__device__ __forceinline__ float les_sqrt(float x) { return sqrt_approx(x); }
__device__ __forceinline__ float les_rcp(float x) { return rcp_approx(x); }
__device__ __forceinline__ double les_sqrt(double x) { return ::sqrt(x); }
__device__ __forceinline__ double les_rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ F2 les_sqrt(F2 x) { return F2(sqrt_approx(x.v.x), sqrt_approx(x.v.y)); }
__device__ __forceinline__ F2 les_rcp(F2 x) { return F2(rcp_approx(x.v.x), rcp_approx(x.v.y)); }

// scalar type of the parameters (and of per-row quantities) for an arithmetic type
template <class R> struct Scalar { using T = R; };
template <> struct Scalar<F2> { using T = float; };
template <class R> using scalar_t = typename Scalar<R>::T;

// Compile-time features of a kernel variant: walls present, eddy viscosity, per-cell force
// field, and the less common forms (factorized attractor / reduced compressibility) read from
// Params at run time. SIMPLE: no force anywhere (sigma = 0 at every order) and
// omega_3 = omega_4 = 1, so every moment of order >= 3 leaves the collision at its attractor
// and the pre-collision moments of those orders are never needed (the compiler drops them).
// UNIT: a forced flow with omega_3 = omega_4 = 1, so that every moment of order >= 3 leaves the
// collision as its attractor plus the source term (the same values the general relaxation
// gives at unit rates, with its multiplications by 1 - omega and omega left out); with GEN the
// attractor is the factorized one where the parameters select it.
// FX: a UNIT collision whose force is uniform with F_y = F_z = 0 (a flow driven along x, as in
// a channel): the source recursion keeps only its x terms, and the moments without an x
// exponent get no source. The same values as UNIT (the terms left out are products with zero).
// BIG: 64-bit element offsets (grids with Q * S >= 2^32).
// FACT / RED: the factorized attractor (Sec. 13) / reduced compressibility (Sec. 12) fixed at
// compile time instead of read from the parameters as GEN does (for SIMPLE collisions, the
// unforced flows the two forms are most often run on).
template <bool WALLS_, bool LES_, bool FIELD_, bool GEN_, bool SIMPLE_ = false, bool UNIT_ = false, bool BIG_ = false,
          bool FX_ = false, bool FACT_ = false, bool RED_ = false>
struct Feat {
    static constexpr bool WALLS = WALLS_, LES = LES_, FIELD = FIELD_, GEN = GEN_, SIMPLE = SIMPLE_, UNIT = UNIT_, BIG = BIG_,
                          FX = FX_, FACT = FACT_, RED = RED_;
    static_assert(!SIMPLE_ || (!FIELD_ && !GEN_), "SIMPLE excludes force fields and the general forms");
    static_assert(!UNIT_ || !SIMPLE_, "UNIT is a forced collision");
    static_assert(!FX_ || (UNIT_ && !FIELD_ && !GEN_), "FX is a UNIT collision with a uniform force along x");
    static_assert(!(FACT_ || RED_) || (SIMPLE_ && !GEN_), "FACT / RED are SIMPLE collisions of one form");
};

// ------------------------------------------------------------------------------------------
// Lattices
// ------------------------------------------------------------------------------------------
template <int D> struct Lat;

template <> struct Lat<3> {
    static constexpr int Q = 27;
    static constexpr int NZ = 3;
    __host__ __device__ static constexpr int ex(int i) { return i % 3 - 1; }
    __host__ __device__ static constexpr int ey(int i) { return (i / 3) % 3 - 1; }
    __host__ __device__ static constexpr int ez(int i) { return i / 9 - 1; }
    __host__ __device__ static constexpr int opp(int i) { return 26 - i; }
};

// Paper's D2Q9 numbering (Sec. 2).
template <> struct Lat<2> {
    static constexpr int Q = 9;
    static constexpr int NZ = 1;
    __host__ __device__ static constexpr int ex(int i) {
        return i == 1 ? 1 : i == 3 ? -1 : i == 5 ? 1 : i == 6 ? -1 : i == 7 ? -1 : i == 8 ? 1 : 0;
    }
    __host__ __device__ static constexpr int ey(int i) {
        return i == 2 ? 1 : i == 4 ? -1 : i == 5 ? 1 : i == 6 ? 1 : i == 7 ? -1 : i == 8 ? -1 : 0;
    }
    __host__ __device__ static constexpr int ez(int) { return 0; }
    __host__ __device__ static constexpr int opp(int i) {
        return i == 0 ? 0 : i <= 4 ? ((i + 1) % 4 + 1) : ((i - 5 + 2) % 4 + 5);
    }
};

template <int D> __host__ __device__ constexpr int slot(int i) {
    return (Lat<D>::ex(i) + 1) + 3 * (Lat<D>::ey(i) + 1) + (D == 3 ? 9 * (Lat<D>::ez(i) + 1) : 0);
}
template <int D> constexpr bool slots_valid() {
    bool seen[27] = {};
    for (int i = 0; i < Lat<D>::Q; ++i) {
        const int t = slot<D>(i);
        if (t < 0 || t >= Lat<D>::Q || seen[t]) return false;
        seen[t] = true;
        if (Lat<D>::opp(Lat<D>::opp(i)) != i) return false;
        if (Lat<D>::ex(Lat<D>::opp(i)) != -Lat<D>::ex(i) || Lat<D>::ey(Lat<D>::opp(i)) != -Lat<D>::ey(i)) return false;
    }
    return true;
}
static_assert(slots_valid<2>() && slots_valid<3>(), "direction tables");

__host__ __device__ constexpr double w1(int e) { return e == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }
template <int D> __host__ __device__ constexpr double weight(int i) {
    return w1(Lat<D>::ex(i)) * w1(Lat<D>::ey(i)) * (D == 3 ? w1(Lat<D>::ez(i)) : 1.0);
}
template <int D> __host__ __device__ constexpr double inv_weight(int i) { return 1.0 / weight<D>(i); }
// weight of tensor slot t = (e_x + 1) + 3 (e_y + 1) + 9 (e_z + 1)
template <int D> __host__ __device__ constexpr double weight_slot(int t) {
    return w1(t % 3 - 1) * w1(t / 3 % 3 - 1) * (D == 3 ? w1(t / 9 - 1) : 1.0);
}

__host__ __device__ constexpr int ord(int t) { return t % 3 + (t / 3) % 3 + t / 9; }
__host__ __device__ constexpr int ex_a(int t) { return t % 3; }
__host__ __device__ constexpr int ex_b(int t) { return (t / 3) % 3; }
__host__ __device__ constexpr int ex_c(int t) { return t / 9; }
__host__ __device__ constexpr int midx(int a, int b, int c) { return a + 3 * b + 9 * c; }
__host__ __device__ constexpr double third_pow(int n) { return n == 0 ? 1.0 : n == 1 ? 1.0 / 3.0 : n == 2 ? 1.0 / 9.0 : 1.0 / 27.0; }

// ------------------------------------------------------------------------------------------
// Storage codec: d = fbar / w - 1 stored as S; arithmetic type R
// ------------------------------------------------------------------------------------------
// Read-only global loads with a 256-byte L2 prefetch hint: the pulled rows are streamed once,
// and fetching whole 256 B blocks measured 1.5 % faster for FP32 storage at 256^3 (no change
// for 16-bit storage, which is issue bound).
__device__ __forceinline__ double ld_stream(const double* p) {
    double v;
    asm("ld.global.nc.L2::256B.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ float ld_stream(const float* p) {
    float v;
    asm("ld.global.nc.L2::256B.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ unsigned short ld_stream(const unsigned short* p) {
    unsigned short v;
    asm("ld.global.nc.L2::256B.b16 %0, [%1];" : "=h"(v) : "l"(p));
    return v;
}

__device__ __forceinline__ unsigned ld_stream(const unsigned* p) {
    unsigned v;
    asm("ld.global.nc.L2::256B.b32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ float2 ld_stream(const float2* p) {
    float2 v;
    asm("ld.global.nc.L2::256B.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
    return v;
}

// ld / st: one entry; ld2 / st2 (FP32 and 16-bit storage): the entries p[0], p[1] of two
// adjacent cells in one access (p must be aligned to two entries), rounded as ld / st round
template <class S> struct Codec;
template <> struct Codec<double> {
    using R = double;
    static __device__ __forceinline__ R ld(const double* p) { return ld_stream(p); }
    static __device__ __forceinline__ R ld_shared(const double* p) { return *p; }
    static __device__ __forceinline__ void st(double* p, R v) { *p = v; }
};
template <> struct Codec<float> {
    using R = float;
    static __device__ __forceinline__ R ld(const float* p) { return ld_stream(p); }
    static __device__ __forceinline__ R ld_shared(const float* p) { return *p; }
    static __device__ __forceinline__ void st(float* p, R v) { *p = v; }
    static __device__ __forceinline__ float2 ld2(const float* p) { return ld_stream(reinterpret_cast<const float2*>(p)); }
    static __device__ __forceinline__ void st2(float* p, float a, float b) { *reinterpret_cast<float2*>(p) = make_float2(a, b); }
};
template <> struct Codec<__nv_bfloat16> {
    using R = float;
    static __device__ __forceinline__ R ld(const __nv_bfloat16* p) {
        return __bfloat162float(__ushort_as_bfloat16(ld_stream(reinterpret_cast<const unsigned short*>(p))));
    }
    static __device__ __forceinline__ R ld_shared(const __nv_bfloat16* p) {
        return __bfloat162float(__ushort_as_bfloat16(*reinterpret_cast<const unsigned short*>(p)));
    }
    static __device__ __forceinline__ void st(__nv_bfloat16* p, R v) { *p = __float2bfloat16_rn(v); }
    static __device__ __forceinline__ float2 ld2(const __nv_bfloat16* p) {
        const unsigned v = ld_stream(reinterpret_cast<const unsigned*>(p));   // BF16 = top half of an FP32
        return make_float2(__uint_as_float(v << 16), __uint_as_float(v & 0xffff0000u));
    }
    static __device__ __forceinline__ void st2(__nv_bfloat16* p, float a, float b) {
        *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(a, b);
    }
};
template <> struct Codec<__half> {
    using R = float;
    static __device__ __forceinline__ R ld(const __half* p) {
        return __half2float(__ushort_as_half(ld_stream(reinterpret_cast<const unsigned short*>(p))));
    }
    static __device__ __forceinline__ R ld_shared(const __half* p) {
        return __half2float(__ushort_as_half(*reinterpret_cast<const unsigned short*>(p)));
    }
    static __device__ __forceinline__ void st(__half* p, R v) { *p = __float2half_rn(v); }
    static __device__ __forceinline__ float2 ld2(const __half* p) {
        const unsigned v = ld_stream(reinterpret_cast<const unsigned*>(p));
        return __half22float2(*reinterpret_cast<const __half2*>(&v));
    }
    static __device__ __forceinline__ void st2(__half* p, float a, float b) {
        *reinterpret_cast<__half2*>(p) = __floats2half2_rn(a, b);
    }
};

// ------------------------------------------------------------------------------------------
// One-dimensional central-moment transforms on (e = -1, 0, +1) populations
// ------------------------------------------------------------------------------------------
// forward: (f-, f0, f+) -> (m0, m1, m2) with m_k = sum f (e - u)^k; u2 = u*u, tu = 2u
// (nu = -u, ntu = -2u: the negations are hoisted out of the nine lines of a sweep)
template <class R> __device__ __forceinline__ void fwd1(R& a, R& b, R& c, R nu, R ntu, R u2) {
    const R s1 = c - a;
    const R s2 = c + a;
    const R m0 = s2 + b;
    a = m0;
    b = fma(nu, m0, s1);
    c = fma(u2, m0, fma(ntu, s1, s2));
}
// the same on populations weighted by the relative 1D weights (1, 4, 1) of e = (-1, 0, +1):
// m_k = sum r1(e) f (e - u)^k, the sum a multiply-add by 4 in place of an add
template <class R> __device__ __forceinline__ void fwd1r(R& a, R& b, R& c, R nu, R ntu, R u2) {
    const R s1 = c - a;
    const R s2 = c + a;
    const R m0 = fma(R(4), b, s2);
    a = m0;
    b = fma(nu, m0, s1);
    c = fma(u2, m0, fma(ntu, s1, s2));
}
// inverse: (m0, m1, m2) -> (2 f-, f0, 2 f+) with the raw moments r1 = sum f e, r2 = sum f e^2:
// f+- = (r2 +- r1) / 2 and f0 = m0 - r2. The halving is left out: the outputs for e = -+1 come
// out doubled, exactly (a power of two commutes with rounding), and the sweeps that follow are
// linear, so the factor travels with them to the last sweep, whose per-line constants absorb it.
template <class R> __device__ __forceinline__ void inv1x2(R& a, R& b, R& c, R u, R tu, R u2) {
    const R m0 = a, m1 = b, m2 = c;
    const R r1 = fma(u, m0, m1);
    const R r2 = fma(u2, m0, fma(tu, m1, m2));
    a = r2 - r1;
    b = m0 - r2;
    c = r2 + r1;
}

// e_i . u_w of direction i with the wall velocity w, the zero components of e_i left out at
// compile time (the compiler keeps a product by zero: it could change the sign of a zero sum)
template <int D, int i, class R> __device__ __forceinline__ R e_dot(const R (&w)[3]) {
    constexpr int ex = Lat<D>::ex(i), ey = Lat<D>::ey(i), ez = Lat<D>::ez(i);
    static_assert(ex != 0 || ey != 0 || ez != 0, "the rest population crosses no wall");
    R r = R(0);
    if constexpr (ex != 0) r = ex > 0 ? w[0] : -w[0];
    if constexpr (ey != 0) {
        if constexpr (ex != 0) r = ey > 0 ? r + w[1] : r - w[1];
        else r = ey > 0 ? w[1] : -w[1];
    }
    if constexpr (ez != 0) {
        if constexpr (ex != 0 || ey != 0) r = ez > 0 ? r + w[2] : r - w[2];
        else r = ez > 0 ? w[2] : -w[2];
    }
    return r;
}
// 6 / (number of walls a link crosses: 1, 2 at an edge, 3 at a corner) of the moving-wall term
template <class R> __device__ __forceinline__ R wall_factor(int cnt) {
    return cnt >= 3 ? R(2) : cnt == 2 ? R(3) : R(6);
}

// ------------------------------------------------------------------------------------------
// Pull with periodic wrap and half-way bounce-back; fills h (slot order) with the deviation
// populations h = w d (kPullDev), the stored deviations d themselves (kPullStored), or the
// populations fbar = w (1 + d) (kPullFull)
// ------------------------------------------------------------------------------------------
enum { kPullStored = 0, kPullDev = 1, kPullFull = 2 };
template <int D, class S, bool WALLS, bool BIG = false, int PULL = kPullDev>
__device__ __forceinline__ void gather_impl(const S* __restrict__ src, int x, int y, int z, const PR<typename Codec<S>::R>& p,
                                       typename Codec<S>::R (&h)[Lat<D>::Q]) {
    using R = typename Codec<S>::R;
    using IX = Ix<BIG>;
    // Q * S < 2^32 is checked at create for the 32-bit variant. On a slab, row offsets of the
    // ghost plane below are negative; they only occur for e_z = +1 (directions 18..26), so
    // i * S + row stays >= 0 and the 32-bit unsigned sum is the exact offset.
    const IX PS = plane_stride<BIG>(p);
    int xs[3], ys[3], zs[3];
    bool xo[3] = {false, false, false}, yo[3] = {false, false, false}, zo[3] = {false, false, false};
#pragma unroll
    for (int k = 0; k < 3; ++k) {          // slot k <-> e = k - 1, source coordinate = x - e
        int sx = x + 1 - k, sy = y + 1 - k, sz = z + 1 - k;
        if (sx < 0 || sx >= p.nx) {
            if (!WALLS || p.bc[0] != 1) sx += (sx < 0) ? p.nx : -p.nx;
            else { xo[k] = true; sx = x; }
        }
        if (sy < 0 || sy >= p.ny) {
            if (!WALLS || p.bc[1] != 1) sy += (sy < 0) ? p.ny : -p.ny;
            else { yo[k] = true; sy = y; }
        }
        if constexpr (D == 3) {
            if (sz < 0 || sz >= p.nz) {
                if (!WALLS || p.bc[2] != 1) sz += (sz < 0) ? p.wz : -p.wz;
                else { zo[k] = true; sz = z; }
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
        constexpr R w = (R)weight<D>(i);
        if constexpr (WALLS) {
            // branch-free: the address is selected and the load is unconditional, so the 27 loads
            // issue back to back; the moving-wall term is added only where a wall was crossed
            const bool bx = xo[a], by = yo[b], bz = zo[c];
            const bool bounced = bx || by || bz;
            const IX own = IX(Lat<D>::opp(i)) * PS + cell;
            const IX pulled = IX(i) * PS + row[c][b] + (unsigned)xs[a];
            R d = Codec<S>::ld(src + (bounced ? own : pulled));
            if (p.moving) {
                // half-way bounce-back from a moving wall: d += 6 (e . u_w), averaged over the
                // walls the link crosses
                constexpr int sx = (a == 2) ? 0 : 1, sy = (b == 2) ? 0 : 1, sz = (c == 2) ? 0 : 1;
                R eu = R(0);
                if constexpr (a != 1) eu = bx ? eu + e_dot<D, i>(p.uw[0][sx]) : eu;
                if constexpr (b != 1) eu = by ? eu + e_dot<D, i>(p.uw[1][sy]) : eu;
                if constexpr (c != 1) eu = bz ? eu + e_dot<D, i>(p.uw[2][sz]) : eu;
                d = fma(wall_factor<R>((int)bx + (int)by + (int)bz), eu, d);
            }
            h[slot<D>(i)] = PULL == kPullStored ? d : PULL == kPullDev ? d * w : fma(d, w, w);
        } else {
            const R d = Codec<S>::ld(src + (IX(i) * PS + row[c][b] + (unsigned)xs[a]));
            h[slot<D>(i)] = PULL == kPullStored ? d : PULL == kPullDev ? d * w : fma(d, w, w);
        }
    });
}

// Pull for a cell: the wall-aware version only where a link can cross a wall (cells in the first
// or last layer of a bounce-back axis); everywhere else the periodic pull, which never leaves the
// box on a wall axis there. With x-rows per warp, y and z are warp-uniform, so the branch only
// diverges on x walls.
template <int D, class S, bool WALLS, bool BIG = false, int PULL = kPullDev>
__device__ __forceinline__ void gather(const S* __restrict__ src, int x, int y, int z, const PR<typename Codec<S>::R>& p,
                                       typename Codec<S>::R (&h)[Lat<D>::Q]) {
    if constexpr (WALLS) {
        const bool near = (p.bc[0] == 1 && (x == 0 || x == p.nx - 1)) || (p.bc[1] == 1 && (y == 0 || y == p.ny - 1)) ||
                          (D == 3 && p.bc[2] == 1 && (z == 0 || z == p.nz - 1));
        if (near) gather_impl<D, S, true, BIG, PULL>(src, x, y, z, p, h);
        else gather_impl<D, S, false, BIG, PULL>(src, x, y, z, p, h);
    } else {
        gather_impl<D, S, false, BIG, PULL>(src, x, y, z, p, h);
    }
}

// ------------------------------------------------------------------------------------------
// Hydrodynamic fields from deviation populations (Eqs. densitycalculation, velocitycalculation)
// ------------------------------------------------------------------------------------------
template <int D, class R> struct Hydro {
    R drho, jx, jy, jz, ux, uy, uz;
};

template <int D, class R, bool GEN = true, bool FORCED = true>
__device__ __forceinline__ Hydro<D, R> hydro(const R (&h)[Lat<D>::Q], const R F[3], const PR<scalar_t<R>>& p) {
    constexpr int NL = Lat<D>::Q / 3;
    Hydro<D, R> o;
    R s0[NL];
    R drho = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        s0[l] = h[3 * l] + h[3 * l + 1] + h[3 * l + 2];
        drho += s0[l];
        jx += h[3 * l + 2] - h[3 * l];
    }
#pragma unroll
    for (int c = 0; c < NL / 3; ++c) jy += s0[3 * c + 2] - s0[3 * c];
    if constexpr (D == 3) {
#pragma unroll
        for (int b = 0; b < 3; ++b) jz += s0[6 + b] - s0[b];
    }
    o.drho = drho;
    if constexpr (FORCED) {
        o.jx = fma(R(0.5), F[0], jx);
        o.jy = fma(R(0.5), F[1], jy);
        o.jz = fma(R(0.5), F[2], jz);
    } else {
        o.jx = jx;
        o.jy = jy;
        o.jz = jz;
    }
    const R inv = rcp((GEN && p.reduced) ? R(p.rho0) : R(1) + drho);
    o.ux = o.jx * inv;
    o.uy = o.jy * inv;
    o.uz = (D == 3) ? o.jz * inv : R(0);
    return o;
}

// The collision reads the stored deviations d = h / w. The weights are products of the 1D
// weights w1(e) = r1(e) / 6 with r1 = (1, 4, 1) for e = (-1, 0, +1), so every moment of h is
// 6^-D times the same moment of r d, r = prod r1. The sweeps below weight by r1 (a multiply-add
// by 4 in place of an add: no product per population), and the collision applies 6^-D where
// it reads a moment (moment_scale).
template <int D> __host__ __device__ constexpr double moment_scale() { return D == 3 ? 1.0 / 216.0 : 1.0 / 36.0; }

// The first pass: the r1-weighted raw moments of every x-line (three deviations with
// e_x = -1, 0, +1): (sum r1 d, sum r1 d e_x, sum r1 d e_x^2), in place. The hydrodynamic fields
// are sums of these, and the x-sweep of the central transform continues from them.
template <int D, class R> __device__ __forceinline__ void raw_x(R (&m)[Lat<D>::Q]) {
    constexpr int NL = Lat<D>::Q / 3;
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        const R a = m[3 * l], b = m[3 * l + 1], c = m[3 * l + 2];
        const R s1 = c - a, s2 = c + a;
        m[3 * l] = fma(R(4), b, s2);
        m[3 * l + 1] = s1;
        m[3 * l + 2] = s2;
    }
}

// rho - 1 and the momentum (Eqs. densitycalculation, velocitycalculation) from the x-line
// moments of raw_x(): line l = (e_y + 1) + 3 (e_z + 1) carries the weight r1(e_y) r1(e_z), so
// the sums over e_y (per e_z) and then over e_z are again multiply-adds by 4
template <int D, class R, bool GEN = true, bool FORCED = true, bool FYZ = true, bool RED = false>
__device__ __forceinline__ Hydro<D, R> hydro_x(const R (&m)[Lat<D>::Q], const R F[3], const PR<scalar_t<R>>& p) {
    using T = scalar_t<R>;
    constexpr int NZ = Lat<D>::NZ;
    const R C = R((T)moment_scale<D>());
    R A[NZ], B[NZ], Y[NZ];
#pragma unroll
    for (int c = 0; c < NZ; ++c) {
        const int l0 = 3 * c, l1 = 3 * c + 1, l2 = 3 * c + 2;      // e_y = -1, 0, +1
        A[c] = fma(R(4), m[3 * l1], m[3 * l0] + m[3 * l2]);
        B[c] = fma(R(4), m[3 * l1 + 1], m[3 * l0 + 1] + m[3 * l2 + 1]);
        Y[c] = m[3 * l2] - m[3 * l0];
    }
    R drho, jx, jy, jz = R(0);
    if constexpr (D == 3) {
        drho = fma(R(4), A[1], A[0] + A[2]);
        jx = fma(R(4), B[1], B[0] + B[2]);
        jy = fma(R(4), Y[1], Y[0] + Y[2]);
        jz = (A[2] - A[0]) * C;
    } else {
        drho = A[0];
        jx = B[0];
        jy = Y[0];
    }
    drho = drho * C;
    jx = jx * C;
    jy = jy * C;
    Hydro<D, R> o;
    o.drho = drho;
    if constexpr (FORCED) {
        o.jx = fma(R(0.5), F[0], jx);
        o.jy = FYZ ? fma(R(0.5), F[1], jy) : jy;
        o.jz = FYZ ? fma(R(0.5), F[2], jz) : jz;
    } else {
        o.jx = jx;
        o.jy = jy;
        o.jz = jz;
    }
    const R inv = rcp(RED || (GEN && p.reduced) ? R(p.rho0) : R(1) + drho);
    o.ux = o.jx * inv;
    o.uy = o.jy * inv;
    o.uz = (D == 3) ? o.jz * inv : R(0);
    return o;
}

// Forward sweeps: deviation populations (slot order) -> central moments of h about u.
template <int D, class R>
__device__ __forceinline__ void central_forward(R (&m)[Lat<D>::Q], R ux, R uy, R uz) {
    constexpr int NL = Lat<D>::Q / 3;
    const R nx = -ux, ny = -uy, nz = -uz;
    const R tx = nx + nx, ty = ny + ny, tz = nz + nz, qx = ux * ux, qy = uy * uy, qz = uz * uz;
#pragma unroll
    for (int l = 0; l < NL; ++l) fwd1(m[3 * l], m[3 * l + 1], m[3 * l + 2], nx, tx, qx);
#pragma unroll
    for (int c = 0; c < Lat<D>::NZ; ++c)
#pragma unroll
        for (int a = 0; a < 3; ++a) fwd1(m[9 * c + a], m[9 * c + 3 + a], m[9 * c + 6 + a], ny, ty, qy);
    if constexpr (D == 3) {
#pragma unroll
        for (int t = 0; t < 9; ++t) fwd1(m[t], m[9 + t], m[18 + t], nz, tz, qz);
    }
}

// The forward transform continued from the raw x-line moments of raw_x(): shift the x-moments
// to central ones about u_x, (m0, s1, s2) -> (m0, s1 - u m0, s2 - 2u s1 + u^2 m0), then the
// y and z sweeps (r1-weighted): 6^D times central_forward() on the populations h = w d.
template <int D, class R>
__device__ __forceinline__ void central_forward_from_x(R (&m)[Lat<D>::Q], R ux, R uy, R uz) {
    constexpr int NL = Lat<D>::Q / 3;
    const R nx = -ux, ny = -uy, nz = -uz;
    const R tx = nx + nx, ty = ny + ny, tz = nz + nz, qx = ux * ux, qy = uy * uy, qz = uz * uz;
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        const R m0 = m[3 * l], s1 = m[3 * l + 1], s2 = m[3 * l + 2];
        m[3 * l + 1] = fma(nx, m0, s1);
        m[3 * l + 2] = fma(qx, m0, fma(tx, s1, s2));
    }
#pragma unroll
    for (int c = 0; c < Lat<D>::NZ; ++c)
#pragma unroll
        for (int a = 0; a < 3; ++a) fwd1r(m[9 * c + a], m[9 * c + 3 + a], m[9 * c + 6 + a], ny, ty, qy);
    if constexpr (D == 3) {
#pragma unroll
        for (int t = 0; t < 9; ++t) fwd1r(m[t], m[9 + t], m[18 + t], nz, tz, qz);
    }
}

// Inverse sweeps: central moments about u -> populations (slot order). Every sweep leaves out
// the halving of f-+ = (r2 -+ r1) / 2 (inv1x2), so that the x-line l = (e_y + 1) + 3 (e_z + 1)
// arrives scaled by 2^k, k = |e_y| + |e_z|. What the last (x) sweep returns, by OUT:
//   kInvPlain:  the populations h (its constants carry 1/2 and 2^-k);
//   kInvDev:    the deviations d = h / w (the inverse weights folded into those constants);
//   kInvScaled: 2^n h with n = |e_x| + |e_y| + |e_z| (no constants at all), for a caller that
//               multiplies every population by a constant anyway (inv_weight_scaled below).
// Each is bitwise the result of halving in every sweep (a power of two commutes with rounding).
enum { kInvPlain = 0, kInvDev = 1, kInvScaled = 2 };
template <int D, class R, int OUT>
__device__ __forceinline__ void central_inverse_impl(R (&m)[Lat<D>::Q], R ux, R uy, R uz) {
    using T = scalar_t<R>;
    constexpr int NL = Lat<D>::Q / 3;
    const R tx = ux + ux, ty = uy + uy, tz = uz + uz, qx = ux * ux, qy = uy * uy, qz = uz * uz;
    if constexpr (D == 3) {
#pragma unroll
        for (int t = 0; t < 9; ++t) inv1x2(m[t], m[9 + t], m[18 + t], uz, tz, qz);
    }
#pragma unroll
    for (int c = 0; c < Lat<D>::NZ; ++c)
#pragma unroll
        for (int a = 0; a < 3; ++a) inv1x2(m[9 * c + a], m[9 * c + 3 + a], m[9 * c + 6 + a], uy, ty, qy);
    if constexpr (OUT == kInvScaled) {
#pragma unroll
        for (int l = 0; l < NL; ++l) inv1x2(m[3 * l], m[3 * l + 1], m[3 * l + 2], ux, tx, qx);
    } else {
        sfor<NL>([&](auto LI) {
            constexpr int l = decltype(LI)::value;
            constexpr int k = (l % 3 != 1) + (l / 3 != 1 && D == 3);
            constexpr double sk = k == 0 ? 1.0 : k == 1 ? 0.5 : 0.25;
            constexpr bool dev = OUT == kInvDev;
            constexpr T he = (T)((dev ? 0.5 / weight_slot<D>(3 * l) : 0.5) * sk),
                        i0 = (T)((dev ? 1.0 / weight_slot<D>(3 * l + 1) : 1.0) * sk);
            const R m0 = m[3 * l], m1 = m[3 * l + 1], m2 = m[3 * l + 2];
            const R r1 = fma(ux, m0, m1);
            const R r2 = fma(qx, m0, fma(tx, m1, m2));
            const R hr2 = r2 * R(he);
            m[3 * l] = fma(R(-he), r1, hr2);
            if constexpr (i0 == T(1)) m[3 * l + 1] = m0 - r2;
            else m[3 * l + 1] = (m0 - r2) * R(i0);
            m[3 * l + 2] = fma(R(he), r1, hr2);
        });
    }
}
template <int D, class R>
__device__ __forceinline__ void central_inverse(R (&m)[Lat<D>::Q], R ux, R uy, R uz) {
    central_inverse_impl<D, R, kInvPlain>(m, ux, uy, uz);
}

// The constant that turns the collision's output for direction i (2^n h, see collide) into the
// stored deviation d = h / w: 1 / (2^n w_i), n = |e_x| + |e_y| + |e_z|.
template <int D> __host__ __device__ constexpr double inv_weight_scaled(int i) {
    const int n = (Lat<D>::ex(i) != 0) + (Lat<D>::ey(i) != 0) + (D == 3 && Lat<D>::ez(i) != 0);
    return inv_weight<D>(i) / double(1 << n);
}

// prod_{d in S}(1/3 + q_d) - 3^{-|S|} without cancellation (all terms are non-negative):
// A_k = (1/3 + q_k) A_{k-1} + q_k 3^{-(k-1)}, A_0 = 0
template <class R, bool X, bool Y, bool Z> __device__ __forceinline__ R excess(const R* q) {
    using T = scalar_t<R>;
    const R third = R(T(1) / 3);
    R A = R(0);
    int k = 0;
    if constexpr (X) { A = q[0]; ++k; }
    if constexpr (Y) { A = (k == 0) ? q[1] : fma(third + q[1], A, q[1] * R(T(1) / 3)); ++k; }
    if constexpr (Z) {
        const T tk = (k == 0) ? T(1) : (k == 1) ? T(1) / 3 : T(1) / 9;
        A = (k == 0) ? q[2] : fma(third + q[2], A, q[2] * R(tk));
    }
    return A;
}

// prod over the axes with a non-zero exponent of cw[d][e_d] (a factor 1 for exponent 0)
template <class R, int a, int b, int c> __device__ __forceinline__ R weight_cm(const R (&cw)[3][3]) {
    R k = R(1);
    bool any = false;
    if constexpr (a > 0) { k = cw[0][a]; any = true; }
    if constexpr (b > 0) { k = any ? k * cw[1][b] : cw[1][b]; any = true; }
    if constexpr (c > 0) { k = any ? k * cw[2][c] : cw[2][c]; }
    return k;
}

// ------------------------------------------------------------------------------------------
// The collision in central-moment space (generic form; see the file header and cmlbm.h).
// In: the stored deviations d = h / w (slot order; h = fbar - w), force F, the eddy-viscosity
// constant cs_eff (0 = off); the weights enter the sweeps as relative factors (raw_x).
// Out: with DEV the post-collision deviations d (the inverse weights folded into the last
// sweep); otherwise the deviation populations h, each scaled by 2^n (n = |e_x| + |e_y| + |e_z|
// of its direction, see central_inverse_impl), which the caller stores as h * inv_weight_scaled.
// R is the arithmetic type (double, float, or F2 for two cells of one row; cs_eff and the
// parameters are then scalars shared by both cells).
// ------------------------------------------------------------------------------------------
template <int D, class R, class FT, bool DEV = false>
__device__ __forceinline__ void collide(R (&m)[Lat<D>::Q], const R F[3], const PR<scalar_t<R>>& p, scalar_t<R> cs_eff) {
    using T = scalar_t<R>;
    constexpr int Q = Lat<D>::Q;
    raw_x<D, R>(m);
    const Hydro<D, R> hy = hydro_x<D, R, FT::GEN, !FT::SIMPLE, !FT::FX, FT::RED>(m, F, p);
    const R drho = hy.drho, rho = R(1) + hy.drho, ndrho = -hy.drho;
    const R u[3] = {hy.ux, hy.uy, hy.uz};
    central_forward_from_x<D, R>(m, u[0], u[1], u[2]);
    const R C = R((T)moment_scale<D>());        // m holds 6^D times the central moments of h
    // zeroth and first order leave the collision at once (their pre-collision central moments
    // are not read): the density deviation, and the momentum plus the source sigma_x = F_x
    // (collision invariants), as central moments about u
    m[0] = drho;
    if constexpr (FT::SIMPLE) {
        m[midx(1, 0, 0)] = fma(ndrho, u[0], hy.jx);
        m[midx(0, 1, 0)] = fma(ndrho, u[1], hy.jy);
        if constexpr (D == 3) m[midx(0, 0, 1)] = fma(ndrho, u[2], hy.jz);
    } else {
        m[midx(1, 0, 0)] = fma(ndrho, u[0], fma(R(0.5), F[0], hy.jx));
        m[midx(0, 1, 0)] = fma(ndrho, u[1], FT::FX ? hy.jy : fma(R(0.5), F[1], hy.jy));
        if constexpr (D == 3) m[midx(0, 0, 1)] = fma(ndrho, u[2], FT::FX ? hy.jz : fma(R(0.5), F[2], hy.jz));
    }

    const R third = R(T(1) / 3);
    const R q[3] = {u[0] * u[0], u[1] * u[1], u[2] * u[2]};
    const R cw[3][3] = {{R(1), -u[0], third + q[0]},
                        {R(1), -u[1], third + q[1]},
                        {R(1), -u[2], third + q[2]}};
    const R irho = rcp(rho);
    const R Fr[3] = {F[0] * irho, F[1] * irho, F[2] * irho};
    const R Fr2[3] = {Fr[0] + Fr[0], Fr[1] + Fr[1], Fr[2] + Fr[2]};

    // second order: non-equilibrium stress Pi = kappa - c_s^2 rho delta (kappa = kbar at order 2)
    const R Pxx = fma(m[midx(2, 0, 0)], C, fma(ndrho, third, q[0]));
    const R Pyy = fma(m[midx(0, 2, 0)], C, fma(ndrho, third, q[1]));
    const R Pxy = fma(m[midx(1, 1, 0)], C, u[0] * u[1]);
    R Pzz = R(0), Pxz = R(0), Pyz = R(0);
    if constexpr (D == 3) {
        Pzz = fma(m[midx(0, 0, 2)], C, fma(ndrho, third, q[2]));
        Pxz = fma(m[midx(1, 0, 1)], C, u[0] * u[2]);
        Pyz = fma(m[midx(0, 1, 1)], C, u[1] * u[2]);
    }

    R wnu;
    if constexpr (FT::LES) {
        R tau = R(p.tau0);
        if (cs_eff > T(0)) {
            R Q2 = Pxx * Pxx;
            Q2 = fma(Pyy, Pyy, Q2);
            Q2 = fma(Pzz, Pzz, Q2);
            R O2 = Pxy * Pxy;
            O2 = fma(Pxz, Pxz, O2);
            O2 = fma(Pyz, Pyz, O2);
            const R Qn = les_sqrt(fma(R(2), O2, Q2));
            // tau_eff = (tau + sqrt(tau^2 + 18 sqrt(2) C^2 |Pi| / rho)) / 2
            const R k = R(T(25.455844122715710878) * cs_eff * cs_eff);
            tau = R(0.5) * (tau + les_sqrt(fma(tau, tau, k * Qn * irho)));
        }
        wnu = les_rcp(tau);
    } else if constexpr (std::is_same_v<R, double>) {
        // the same value as the reciprocal below (both IEEE-rounded), without an FP64 division
        // per cell on GB300's narrow FP64 pipe; the FP32 forms keep the per-thread reciprocal,
        // which measured faster there (register allocation of the 16-bit steps)
        wnu = R(p.omega_nu);
    } else {
        wnu = rcp(R(p.tau0));
    }
    const R wb = (p.omega_bulk > T(0)) ? R(p.omega_bulk) : wnu;

    // kappa of f at second order, used by the source recursion (sigma = 0 at second order)
    R kap[Q];
    kap[midx(2, 0, 0)] = fma(rho, third, Pxx);
    kap[midx(0, 2, 0)] = fma(rho, third, Pyy);
    kap[midx(1, 1, 0)] = Pxy;
    if constexpr (D == 3) {
        kap[midx(0, 0, 2)] = fma(rho, third, Pzz);
        kap[midx(1, 0, 1)] = Pxz;
        kap[midx(0, 1, 1)] = Pyz;
    }

    // relaxed second order: trace with omega_b, deviator and off-diagonal with omega_nu
    const R tr = Pxx + Pyy + Pzz;
    const R corr = (wnu - wb) * tr * R(T(1) / D);
    const R omn = R(1) - wnu;
    const R Txx = fma(omn, Pxx, corr);
    const R Tyy = fma(omn, Pyy, corr);
    const R Tzz = fma(omn, Pzz, corr);
    const R Txy = omn * Pxy;
    const R Txz = omn * Pxz;
    const R Tyz = omn * Pyz;
    const R w3 = R(p.omega3), w4 = R(p.omega4);
    const R om3 = R(T(1) - p.omega3), om4 = R(T(1) - p.omega4);
    const bool factorized = (FT::GEN && p.attractor != 0) || FT::FACT;

    // the factorized attractor of moment (a, b, c) (Sec. 13: products of the relaxed second-order
    // moments over rho^(k-1)) as a deviation from the weights' moment, where the pattern has a
    // product rule; DM (the Maxwellian one) otherwise
    auto factorized_dm = [&](auto AI, auto BI, auto CI, R DM) -> R {
        constexpr int a = decltype(AI)::value, b = decltype(BI)::value, c = decltype(CI)::value;
        constexpr int ones = (a == 1) + (b == 1) + (c == 1);
        constexpr int twos = (a == 2) + (b == 2) + (c == 2);
        if constexpr (ones == 0) {
            const R pt[3] = {Txx * irho, Tyy * irho, Tzz * irho};
            R prodp = R(1);
            if constexpr (a == 2) prodp = prodp * (third + pt[0]);
            if constexpr (b == 2) prodp = prodp * (third + pt[1]);
            if constexpr (c == 2) prodp = prodp * (third + pt[2]);
            return fma(drho, prodp, excess<R, a == 2, b == 2, c == 2>(pt) - excess<R, a == 2, b == 2, c == 2>(q));
        } else if constexpr (ones == 2 && twos == 1) {
            constexpr int dtwo = (a == 2) ? 0 : (b == 2) ? 1 : 2;
            const R Tdg = dtwo == 0 ? Txx : dtwo == 1 ? Tyy : Tzz;
            const R Toff = (a != 1) ? Tyz : (b != 1) ? Txz : Txy;
            const R uoff = (a != 1) ? u[1] * u[2] : (b != 1) ? u[0] * u[2] : u[0] * u[1];
            return fma(Toff, fma(Tdg, irho, third), -((third + q[dtwo]) * uoff));
        } else {
            return DM;
        }
    };

    if constexpr (FT::SIMPLE) {
        // no source and omega_3 = omega_4 = 1: orders >= 3 are set to their attractors
        sfor<Q>([&](auto TI) {
            constexpr int t = decltype(TI)::value;
            if constexpr (ord(t) >= 3) {
                constexpr int a = ex_a(t), b = ex_b(t), c = ex_c(t);
                constexpr bool even = (a % 2 == 0) && (b % 2 == 0) && (c % 2 == 0);
                R DM;
                if constexpr (even) {
                    const R tp = R((T)third_pow((a == 2) + (b == 2) + (c == 2)));
                    DM = fma(drho, tp, -excess<R, a == 2, b == 2, c == 2>(q));
                } else {
                    DM = -weight_cm<R, a, b, c>(cw);
                }
                if constexpr (FT::FACT)
                    DM = factorized_dm(std::integral_constant<int, a>{}, std::integral_constant<int, b>{},
                                       std::integral_constant<int, c>{}, DM);
                m[t] = DM;
            }
        });
    } else {
        // orders >= 3 in increasing order: source by the hierarchical identity, attractor, relaxation
        sfor<2 * D + 1>([&](auto NI) {
            constexpr int n = decltype(NI)::value;
            sfor<Q>([&](auto TI) {
                constexpr int t = decltype(TI)::value;
                if constexpr (n >= 3 && ord(t) == n) {
                    constexpr int a = ex_a(t), b = ex_b(t), c = ex_c(t);
                    R s = R(0);
                    if constexpr (a > 0) s = fma(a == 2 ? Fr2[0] : Fr[0], kap[t - 1], s);
                    if constexpr (b > 0 && !FT::FX) s = fma(b == 2 ? Fr2[1] : Fr[1], kap[t - 3], s);
                    if constexpr (c > 0 && !FT::FX) s = fma(c == 2 ? Fr2[2] : Fr[2], kap[t - 9], s);
                    constexpr bool sourced = a > 0 || (!FT::FX && (b > 0 || c > 0));
                    const R hs = R(0.5) * s;
                    const R kw = weight_cm<R, a, b, c>(cw);
                    if constexpr (ord(t) < 2 * D) {
                        if constexpr (sourced) kap[t] = fma(R(0.5), s, fma(m[t], C, kw));
                        else kap[t] = fma(m[t], C, kw);
                    }
                    constexpr bool even = (a % 2 == 0) && (b % 2 == 0) && (c % 2 == 0);
                    constexpr int twos = (a == 2) + (b == 2) + (c == 2);
                    const R tp = R((T)third_pow(twos));
                    R DM;
                    if constexpr (even) DM = fma(drho, tp, -excess<R, a == 2, b == 2, c == 2>(q));
                    else DM = -kw;
                    if (factorized)
                        DM = factorized_dm(std::integral_constant<int, a>{}, std::integral_constant<int, b>{},
                                           std::integral_constant<int, c>{}, DM);
                    if constexpr (FT::UNIT) {
                        // fma(0, ., fma(1, DM, hs)) of the general form: DM + s/2 rounded once (the
                        // halving is exact). The standard collision writes it as one packed fma; the
                        // general forms keep the product and the sum, which measured fewer spills
                        // there (0-24 B against 16-44 B at 128 registers, FP32)
                        if constexpr (!sourced) m[t] = DM;
                        else if constexpr (FT::GEN) m[t] = DM + hs;
                        else m[t] = fma(R(0.5), s, DM);
                    } else {
                        const R w = (ord(t) == 3) ? w3 : w4;
                        const R om = (ord(t) == 3) ? om3 : om4;
                        m[t] = fma(om, fma(m[t], C, hs), fma(w, DM, hs));
                    }
                }
            });
        });
    }

    // second order back to deviations of the weights' moments
    m[midx(2, 0, 0)] = Txx + fma(drho, third, -q[0]);
    m[midx(0, 2, 0)] = Tyy + fma(drho, third, -q[1]);
    m[midx(1, 1, 0)] = fma(-u[0], u[1], Txy);
    if constexpr (D == 3) {
        m[midx(0, 0, 2)] = Tzz + fma(drho, third, -q[2]);
        m[midx(1, 0, 1)] = fma(-u[0], u[2], Txz);
        m[midx(0, 1, 1)] = fma(-u[1], u[2], Tyz);
    }

    central_inverse_impl<D, R, DEV ? kInvDev : kInvScaled>(m, u[0], u[1], u[2]);
}

// Equilibrium deviations fbar - w for (rho, u, F): central moments kappa^M - sigma^M / 2 about u
template <int D, class R>
__device__ __forceinline__ void equilibrium(R (&m)[Lat<D>::Q], R rho, R ux, R uy, R uz, const R F[3]) {
    constexpr int Q = Lat<D>::Q;
    const R u[3] = {ux, uy, uz};
    const R q[3] = {ux * ux, uy * uy, uz * uz};
    const R cw[3][3] = {{R(1), -u[0], R(1) / 3 + q[0]},
                        {R(1), -u[1], R(1) / 3 + q[1]},
                        {R(1), -u[2], R(1) / 3 + q[2]}};
    const R drho = rho - R(1);
    sfor<Q>([&](auto TI) {
        constexpr int t = decltype(TI)::value;
        constexpr int a = ex_a(t), b = ex_b(t), c = ex_c(t);
        constexpr bool even = (a % 2 == 0) && (b % 2 == 0) && (c % 2 == 0);
        constexpr int twos = (a == 2) + (b == 2) + (c == 2);
        constexpr R tp = (R)third_pow(twos);
        // sigma^M by the identity on the Maxwellian moments: non-zero only for one odd axis
        R s = 0;
        if constexpr (a == 1 && (b % 2 == 0) && (c % 2 == 0)) s += F[0] * tp;
        if constexpr (b == 1 && (a % 2 == 0) && (c % 2 == 0)) s += F[1] * tp;
        if constexpr (c == 1 && (a % 2 == 0) && (b % 2 == 0)) s += F[2] * tp;
        const R kw = cw[0][a] * cw[1][b] * cw[2][c];
        R DM;
        if constexpr (ord(t) == 0) DM = drho;
        else if constexpr (even) DM = drho * tp - excess<R, a == 2, b == 2, c == 2>(q);
        else DM = -kw;
        m[t] = DM - R(0.5) * s;
    });
    central_inverse<D, R>(m, u[0], u[1], u[2]);
}

}  // namespace cm
