// Shared device helpers: small fixed-size vectors of conserved variables,
// Euler physics (Eq. 3 with B = 0), periodic indexing and the device error flag.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define ADER_DEV __host__ __device__ __forceinline__

namespace ader {

// Device error flag bits (turned into ADER_ERR_* by ader_sync_status).
enum : unsigned { FLAG_UNPHYSICAL = 1u, FLAG_NONFINITE = 2u, FLAG_NOT_CONVERGED = 4u };

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

// ------------------------------------------------------------------ Euler physics, Eq. 3
template <class R>
struct Prim {
    R irho, vx, vy, vz, p;
};

template <class R>
ADER_DEV Prim<R> primitives(const Vec<5, R>& u, R gm1) {
    Prim<R> q;
    q.irho = rcp(u[0]);
    q.vx = u[1] * q.irho;
    q.vy = u[2] * q.irho;
    q.vz = u[3] * q.irho;
    q.p = gm1 * (u[4] - R(0.5) * (u[1] * q.vx + u[2] * q.vy + u[3] * q.vz));
    return q;
}

// physical flux in direction D (0: F, 1: G, 2: H)
template <int D, class R>
ADER_DEV Vec<5, R> flux_from(const Vec<5, R>& u, const Prim<R>& q) {
    const R vn = D == 0 ? q.vx : (D == 1 ? q.vy : q.vz);
    Vec<5, R> f;
    f[0] = u[1 + D];
    f[1] = u[1] * vn;
    f[2] = u[2] * vn;
    f[3] = u[3] * vn;
    f[1 + D] += q.p;
    f[4] = (u[4] + q.p) * vn;
    return f;
}

template <int D, class R>
ADER_DEV Vec<5, R> flux(const Vec<5, R>& u, R gm1) {
    return flux_from<D>(u, primitives(u, gm1));
}

// ------------------------------------------------------------------ indexing
struct Grid {
    int nx, ny, nz;
    long long n;      // nx*ny*nz
};

ADER_DEV int wrap(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

// linear index of the zone displaced by (di, dj, dk) from (i, j, k), periodic
ADER_DEV long long nbr(const Grid& g, int i, int j, int k, int di, int dj, int dk) {
    return ((long long)wrap(k + dk, g.nz) * g.ny + wrap(j + dj, g.ny)) * g.nx + wrap(i + di, g.nx);
}

ADER_DEV void raise_flag(unsigned* flag, unsigned bit) {
#ifdef __CUDA_ARCH__
    if (flag) atomicOr(flag, bit);
#else
    if (flag) *flag |= bit;
#endif
}

}  // namespace ader
