// Shared device helpers: small fixed-size vectors of conserved variables,
// Euler physics (Eq. 3 with B = 0), periodic indexing and the device error flag.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define ADER_DEV __host__ __device__ __forceinline__

namespace ader {

// Device error flag bits (turned into ADER_ERR_* by ader_sync_status).
enum : unsigned { FLAG_UNPHYSICAL = 1u, FLAG_NONFINITE = 2u, FLAG_NOT_CONVERGED = 4u, FLAG_TIMEOUT = 8u };

// A vector of NV conserved variables in precision R.  The modal formulas of
// the paper are written on whole vectors, one arithmetic statement for all
// variables; nvcc unrolls everything into registers.
template <int NV, class R>
struct Vec {
    R v[NV];
    ADER_DEV R& operator[](int i) { return v[i]; }
    ADER_DEV const R& operator[](int i) const { return v[i]; }
};

template <int NV, class R>
ADER_DEV Vec<NV, R> operator+(const Vec<NV, R>& a, const Vec<NV, R>& b) {
    Vec<NV, R> r;
#pragma unroll
    for (int i = 0; i < NV; ++i) r.v[i] = a.v[i] + b.v[i];
    return r;
}
template <int NV, class R>
ADER_DEV Vec<NV, R> operator-(const Vec<NV, R>& a, const Vec<NV, R>& b) {
    Vec<NV, R> r;
#pragma unroll
    for (int i = 0; i < NV; ++i) r.v[i] = a.v[i] - b.v[i];
    return r;
}
template <int NV, class R>
ADER_DEV Vec<NV, R> operator-(const Vec<NV, R>& a) {
    Vec<NV, R> r;
#pragma unroll
    for (int i = 0; i < NV; ++i) r.v[i] = -a.v[i];
    return r;
}
template <int NV, class R>
ADER_DEV Vec<NV, R> operator*(double s, const Vec<NV, R>& a) {
    Vec<NV, R> r;
    const R c = R(s);
#pragma unroll
    for (int i = 0; i < NV; ++i) r.v[i] = c * a.v[i];
    return r;
}
template <int NV, class R>
ADER_DEV Vec<NV, R> operator*(const Vec<NV, R>& a, double s) { return s * a; }
template <int NV, class R>
ADER_DEV Vec<NV, R> operator/(const Vec<NV, R>& a, double s) { return (1.0 / s) * a; }
template <int NV, class R>
ADER_DEV Vec<NV, R>& operator+=(Vec<NV, R>& a, const Vec<NV, R>& b) { a = a + b; return a; }
template <int NV, class R>
ADER_DEV Vec<NV, R>& operator-=(Vec<NV, R>& a, const Vec<NV, R>& b) { a = a - b; return a; }
template <int NV, class R>
ADER_DEV Vec<NV, R> vzero() {
    Vec<NV, R> r;
#pragma unroll
    for (int i = 0; i < NV; ++i) r.v[i] = R(0);
    return r;
}
// runtime scalar (not a literal) times a vector, kept in precision R
template <int NV, class R>
ADER_DEV Vec<NV, R> scale(R s, const Vec<NV, R>& a) {
    Vec<NV, R> r;
#pragma unroll
    for (int i = 0; i < NV; ++i) r.v[i] = s * a.v[i];
    return r;
}

template <class R> ADER_DEV R rcp(R x) { return R(1) / x; }

// FP64 reciprocal by Newton-Raphson: the hardware's approximate reciprocal
// seeds r, and two steps of r <- r + r (1 - x r) take it to about one unit in
// the last place (the seed's error squares at each step).  On GB300 the FP64
// units are scarce; this costs one seed and four FMAs instead of a correctly
// rounded division.  Zero, infinite and subnormal arguments do not occur where
// it is used (densities, positive sums of weights and wave-speed spans).
template <> ADER_DEV double rcp<double>(double x) {
#ifdef __CUDA_ARCH__
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    double e = fma(-x, r, 1.0);
    r = fma(r, e, r);
    e = fma(-x, r, 1.0);
    return fma(r, e, r);
#else
    return 1.0 / x;
#endif
}

// ------------------------------------------------------------------ FP32 <-> FP64 without the FP64 units
// GB300 runs FP64 at 1/64 of the FP32 rate and its conversion instructions on the same scarce units, so
// the FP32-bulk kernels move values between the two formats with integer operations on the bit
// patterns (IEEE 754 binary32 and binary64: sign, biased exponent, significand).

// x rounded to the nearest FP32 value (ties to even), as a conversion would round it, except that
// results below FP32's normal range are flushed to a signed zero (the FP32 kernels flush such values
// anyway).  Overflow gives a signed infinity, NaN a quiet NaN.
__device__ __forceinline__ float f32_of_f64(double x) {
    const long long b = __double_as_longlong(x);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const unsigned sign = hi & 0x80000000u;
    const unsigned ef = (hi >> 20) & 0x7ffu;
    const int e = (int)ef - 896;                          // exponent rebased from FP64's bias to FP32's
    const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);
    const unsigned rest = lo & 0x1fffffffu;               // the 29 significand bits dropped
    unsigned bits = sign | ((unsigned)(e > 0 ? e : 0) << 23) | m;
    bits += (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) ? 1u : 0u;   // may carry into inf
    const bool nan = ef == 0x7ffu && ((hi & 0xfffffu) | lo) != 0u;
    bits = e <= 0 ? sign : (e >= 255 ? (sign | 0x7f800000u) : bits);
    return __uint_as_float(nan ? 0x7fc00000u : bits);
}

// the FP64 value of an FP32 number, exactly (FP32 subnormals, flushed by the FP32 kernels, give zero)
__device__ __forceinline__ double f64_of_f32(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned e = (b >> 23) & 0xffu;
    const unsigned ed = e == 0u ? 0u : (e == 0xffu ? 0x7ffu : e + 896u);
    const unsigned mant = e == 0u ? 0u : (b & 0x7fffffu);
    return __hiloint2double((int)((b & 0x80000000u) | (ed << 20) | (mant >> 3)), (int)(mant << 29));
}

// x > 0 for an FP64 argument that is not NaN (tolerances, step sizes), decided on its bit pattern: the
// FP32 kernels then issue no FP64 comparison per zone
ADER_DEV bool positive_arg(double x) {
#ifdef __CUDA_ARCH__
    return __double_as_longlong(x) > 0;
#else
    return x > 0.0;
#endif
}

// an FP64 argument in the bulk precision R (FP32: rounded by integer operations on the device)
template <class R>
ADER_DEV R bulk_arg(double x) {
#ifdef __CUDA_ARCH__
    if constexpr (sizeof(R) == 4) return f32_of_f64(x);
#endif
    return R(x);
}

// ------------------------------------------------------------------ physics, Eq. 3 (Gaussian units)
// NV = 5: Euler (rho, rho v, eps).  NV = 8: ideal MHD (rho, rho v, eps, B) with
// eps = rho v^2/2 + P/(gamma-1) + B^2/(8 pi).
constexpr double INV_FOUR_PI = 0.079577471545947667884;   // 1 / (4 pi)

template <int NV, class R>
struct Prim {
    R irho, vx, vy, vz, p;        // p: gas pressure
    R ptot, vB;                    // MHD: P + B^2/8pi and v.B (unused for Euler)
};

template <int NV, class R>
ADER_DEV Prim<NV, R> primitives(const Vec<NV, R>& u, R gm1) {
    Prim<NV, R> q;
    q.irho = rcp(u[0]);
    q.vx = u[1] * q.irho;
    q.vy = u[2] * q.irho;
    q.vz = u[3] * q.irho;
    const R ke = R(0.5) * (u[1] * q.vx + u[2] * q.vy + u[3] * q.vz);
    if constexpr (NV == 8) {
        const R pm = R(0.5 * INV_FOUR_PI) * (u[5] * u[5] + u[6] * u[6] + u[7] * u[7]);
        q.p = gm1 * (u[4] - ke - pm);
        q.ptot = q.p + pm;
        q.vB = q.vx * u[5] + q.vy * u[6] + q.vz * u[7];
    } else {
        q.p = gm1 * (u[4] - ke);
        q.ptot = q.p;
        q.vB = R(0);
    }
    return q;
}

// physical flux in direction D (0: F, 1: G, 2: H) of Eq. 3
template <int D, int NV, class R>
ADER_DEV Vec<NV, R> flux_from(const Vec<NV, R>& u, const Prim<NV, R>& q) {
    const R vn = D == 0 ? q.vx : (D == 1 ? q.vy : q.vz);
    Vec<NV, R> f;
    f[0] = u[1 + D];
    if constexpr (NV == 8) {
        const R bn = R(INV_FOUR_PI) * u[5 + D];
        f[1] = u[1] * vn - bn * u[5];
        f[2] = u[2] * vn - bn * u[6];
        f[3] = u[3] * vn - bn * u[7];
        f[1 + D] += q.ptot;
        f[4] = (u[4] + q.ptot) * vn - bn * q.vB;
        const R Bn = u[5 + D];
        f[5] = vn * u[5] - q.vx * Bn;
        f[6] = vn * u[6] - q.vy * Bn;
        f[7] = vn * u[7] - q.vz * Bn;
        f[5 + D] = R(0);
    } else {
        f[1] = u[1] * vn;
        f[2] = u[2] * vn;
        f[3] = u[3] * vn;
        f[1 + D] += q.p;
        f[4] = (u[4] + q.p) * vn;
    }
    return f;
}

// the physical flux of one direction from the conserved state; Euler takes only what that direction
// needs (the normal velocity and P = (gamma - 1)(eps - |rho v|^2 / 2 rho), no transverse velocities)
template <int D, int NV, class R>
ADER_DEV Vec<NV, R> flux(const Vec<NV, R>& u, R gm1) {
    if constexpr (NV == 5) {
        const R irho = rcp(u[0]);
        const R vn = u[1 + D] * irho;
        const R m2 = u[1] * u[1] + u[2] * u[2] + u[3] * u[3];
        const R p = gm1 * (u[4] - R(0.5) * irho * m2);
        Vec<NV, R> f;
        f[0] = u[1 + D];
        f[1] = u[1] * vn;
        f[2] = u[2] * vn;
        f[3] = u[3] * vn;
        f[1 + D] += p;
        f[4] = (u[4] + p) * vn;
        return f;
    } else {
        return flux_from<D>(u, primitives(u, gm1));
    }
}

// fast magnetosonic speed in direction D (the sound speed for Euler)
template <int D, int NV, class R>
ADER_DEV R fast_speed(const Vec<NV, R>& u, const Prim<NV, R>& q, R gamma) {
    const R a2 = gamma * q.p * q.irho;
    if constexpr (NV == 8) {
        const R f = R(INV_FOUR_PI) * q.irho;
        const R b2 = f * (u[5] * u[5] + u[6] * u[6] + u[7] * u[7]);
        const R bn2 = f * u[5 + D] * u[5 + D];
        const R s = a2 + b2;
        const R disc = sqrt(fmax(s * s - R(4) * a2 * bn2, R(0)));
        return sqrt(R(0.5) * (s + disc));
    } else {
        return sqrt(a2);
    }
}

// ------------------------------------------------------------------ non-stiff source S(U) of Eq. 4
// The paper carries a general source through every predictor and through
// Eq. 6 without naming one; two models are built.  SOURCE_LINEAR: S = -k U on
// the five hydrodynamic components.  SOURCE_GRAVITY: a uniform acceleration g,
// S = (0, rho g, rho v . g).  The field components of MHD get no source (the
// face field evolves by constrained transport alone).  Src holds the model
// with dt folded in: the predictor works with s = dt S, as with the scaled
// fluxes of Eq. 5.
enum { SOURCE_NONE = 0, SOURCE_LINEAR = 1, SOURCE_GRAVITY = 2 };

template <class R>
struct Src {
    int kind;
    R a[3];           // dt k (linear) or dt g (gravity)
};

template <int NV, class R>
ADER_DEV Vec<NV, R> source_at(const Vec<NV, R>& u, const Src<R>& s) {
    Vec<NV, R> r = vzero<NV, R>();
    if (s.kind == SOURCE_LINEAR) {
#pragma unroll
        for (int v = 0; v < 5; ++v) r[v] = -s.a[0] * u[v];
    } else {
        r[1] = s.a[0] * u[0];
        r[2] = s.a[1] * u[0];
        r[3] = s.a[2] * u[0];
        r[4] = s.a[0] * u[1] + s.a[1] * u[2] + s.a[2] * u[3];
    }
    return r;
}

// ------------------------------------------------------------------ predictor control
// Fixed mode (tol <= 0): exactly n_iter Picard steps (M - 1 in the paper).
// Converged mode (tol > 0): iterate until the largest change of an
// evolutionary mode is below tol * (largest |w_1| of the zone), at most
// max_iter times.  iters / capped report what happened.
struct PredCtl {
    int n_iter;
    double tol;
    int max_iter;
    int iters;
    bool capped;
};

template <int NV, class R>
ADER_DEV R max_abs_diff(const Vec<NV, R>& a, const Vec<NV, R>& b) {
    R m = R(0);
#pragma unroll
    for (int v = 0; v < NV; ++v) m = fmax(m, fabs(a[v] - b[v]));
    return m;
}

template <int NV, class R>
ADER_DEV R max_abs(const Vec<NV, R>& a) {
    R m = R(0);
#pragma unroll
    for (int v = 0; v < NV; ++v) m = fmax(m, fabs(a[v]));
    return m;
}

// ------------------------------------------------------------------ indexing
struct Grid {
    int nx, ny, nz;
    long long n;      // nx*ny*nz
};

// i modulo n in [0, n).  Every caller displaces an in-range coordinate by a
// few zones, so two comparisons decide it; the remainder is the fallback for
// displacements beyond one period (grids thinner than the stencil).
ADER_DEV int wrap(int i, int n) {
    if (i >= 0 && i < n) return i;
    if (i < 0 && i >= -n) return i + n;
    if (i >= n && i < 2 * n) return i - n;
    i %= n;
    return i < 0 ? i + n : i;
}

// (i, j, k) of the linear zone index z (x fastest).  Grids of up to 2^32 zones
// take 32-bit divisions, which cost a fraction of the 64-bit ones.
ADER_DEV void zone_ijk(const Grid& g, long long z, int& i, int& j, int& k) {
    if (g.n <= 0xffffffffLL) {
        const unsigned u = (unsigned)z, nx = (unsigned)g.nx, ny = (unsigned)g.ny;
        const unsigned t = u / nx;
        i = (int)(u - t * nx);
        const unsigned q = t / ny;
        j = (int)(t - q * ny);
        k = (int)q;
    } else {
        i = (int)(z % g.nx);
        const long long t = z / g.nx;
        j = (int)(t % g.ny);
        k = (int)(t / g.ny);
    }
}

// linear index of the zone displaced by (di, dj, dk) from (i, j, k), periodic
ADER_DEV long long nbr(const Grid& g, int i, int j, int k, int di, int dj, int dk) {
    return ((long long)wrap(k + dk, g.nz) * g.ny + wrap(j + dj, g.ny)) * g.nx + wrap(i + di, g.nx);
}

// linear index of the zone o zones from zone z = (i, j, k) along direction d, periodic
ADER_DEV long long nbr_along(const Grid& g, long long z, int i, int j, int k, int d, int o) {
    if (d == 0) return z + (wrap(i + o, g.nx) - i);
    if (d == 1) return z + (long long)(wrap(j + o, g.ny) - j) * g.nx;
    return z + (long long)(wrap(k + o, g.nz) - k) * ((long long)g.nx * g.ny);
}

ADER_DEV void raise_flag(unsigned* flag, unsigned bit) {
#ifdef __CUDA_ARCH__
    if (flag) atomicOr(flag, bit);
#else
    if (flag) *flag |= bit;
#endif
}

}  // namespace ader
