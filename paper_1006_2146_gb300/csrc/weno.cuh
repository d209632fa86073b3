// WENO building blocks of the zone-centred reconstruction (see recon.cu for the reading).
#pragma once
#include "common.cuh"

namespace ader {

constexpr double WENO_EPS = 1.0e-12;

template <class R>
ADER_DEV R wsq(R is, R eps) {
    const R t = eps + is;
    return t * t;
}

// Unnormalised nonlinear weights a[s] and their normaliser inv, such that the
// blend is (sum_s a[s] x_s) * inv = sum_s w_s x_s with
// w_s = (g_s / q_s) / sum_r (g_r / q_r), q = (eps + IS)^2.
// FP64 clears the denominators, a[s] = g_s prod_{r != s} q_r: one division
// per blend instead of S + 1.  Every q is at least 1e-24, so the products of
// up to three of them stay far inside the FP64 range.  FP32 keeps the quotient
// form, where such products would underflow.  g may be any positive multiple
// of the linear weights: the normalisation removes it.
template <int S, class R>
ADER_DEV R weno_weights(const R* g, const R* is, R* a, R eps = R(WENO_EPS)) {
    if constexpr (sizeof(R) == 8) {
        R q[S], pre[S], suf[S];
#pragma unroll
        for (int s = 0; s < S; ++s) q[s] = wsq(is[s], eps);
        pre[0] = R(1);
#pragma unroll
        for (int s = 1; s < S; ++s) pre[s] = pre[s - 1] * q[s - 1];
        suf[S - 1] = R(1);
#pragma unroll
        for (int s = S - 2; s >= 0; --s) suf[s] = suf[s + 1] * q[s + 1];
        R d = R(0);
#pragma unroll
        for (int s = 0; s < S; ++s) {
            a[s] = g[s] * (pre[s] * suf[s]);
            d += a[s];
        }
        return rcp(d);
    } else {
        R d = R(0);
#pragma unroll
        for (int s = 0; s < S; ++s) {
            a[s] = g[s] / wsq(is[s], eps);
            d += a[s];
        }
        return rcp(d);
    }
}

// order-3 1-D WENO on the five values a[-2..2] (a[2] = centre); returns b, c.
// Each candidate is carried doubled, B = 2b and C = 2c, built from the four
// neighbour differences d1..d4 (ten operations for the six moments), and the
// smoothness indicators are 4 IS = B^2 + 13/3 C^2 with 4 EPS: every (EPS + IS)^2
// is scaled by the same 16, so the normalised weights are unchanged.
template <class R>
ADER_DEV void weno3_doubled(const R* a, R* al, R& inv, R* B, R* C) {
    const R d1 = a[1] - a[0], d2 = a[2] - a[1], d3 = a[3] - a[2], d4 = a[4] - a[3];
    B[0] = R(3) * d2 - d1;  C[0] = d2 - d1;              // stencil {i-2, i-1, i}
    B[1] = d2 + d3;         C[1] = d3 - d2;              // {i-1, i, i+1}
    B[2] = R(3) * d3 - d4;  C[2] = d4 - d3;              // {i, i+1, i+2}
    const R k13 = R(13.0 / 3.0);
    const R g[3] = {R(1), R(10), R(1)};                  // (1, 10, 1) / 12
    R is[3];
#pragma unroll
    for (int s = 0; s < 3; ++s) is[s] = B[s] * B[s] + k13 * (C[s] * C[s]);
    inv = weno_weights<3>(g, is, al, R(4.0 * WENO_EPS));
}

// ---------------------------------------------------------------- FP64: order 3 from per-position terms
// Along one direction, with w(p) the field at position p:
//   d(p)  = w(p) - w(p-1)                   the difference at face p - 1/2,
//   D2(p) = d(p+1) - d(p)                   the doubled C of the stencil centred on p,
//   E(p)  = 4 EPS + (13/3) D2(p)^2          the C part of 4 (EPS + IS) of that stencil.
// Zone j's candidates are the stencils centred on j-1, j and j+1: doubled slopes B0 = 3 d(j) - d(j-1),
// B1 = d(j) + d(j+1), B2 = 3 d(j+1) - d(j+2), doubled curvatures D2(j-1..j+1), and 4 (EPS + IS_s) =
// B_s^2 + E(j-1+s).  d, D2 and E belong to positions, not zones: a tile computes each once for the four
// (or three) zones that use it (k_cross1_tiled64), and the per-zone form below takes them from the five
// values with the same operations, so the two give the same bits.  The weights clear their denominators
// as weno_weights does: (1, 10, 1) times the product of the other two (EPS + IS)^2.
// Every operation of this form is explicitly rounded (no multiply-add contraction left to the compiler),
// so that the tile and the per-zone kernel, compiled apart, round every step alike.  (Other scalar types,
// such as the host FLOP counter's, take the plain operators.)
template <class R> ADER_DEV R rn_add(R x, R y) { return x + y; }
template <class R> ADER_DEV R rn_sub(R x, R y) { return x - y; }
template <class R> ADER_DEV R rn_mul(R x, R y) { return x * y; }
template <> ADER_DEV double rn_add<double>(double x, double y) {
#ifdef __CUDA_ARCH__
    return __dadd_rn(x, y);
#else
    return x + y;
#endif
}
template <> ADER_DEV double rn_sub<double>(double x, double y) {
#ifdef __CUDA_ARCH__
    return __dsub_rn(x, y);
#else
    return x - y;
#endif
}
template <> ADER_DEV double rn_mul<double>(double x, double y) {
#ifdef __CUDA_ARCH__
    return __dmul_rn(x, y);
#else
    return x * y;
#endif
}

template <class R>
ADER_DEV R w3_curv(R D2) { return fma(rn_mul(R(13.0 / 3.0), D2), D2, R(4.0 * WENO_EPS)); }

template <bool WANT_C, class R>
ADER_DEV void weno3_terms(const R* d, const R* E, const R* D2, R& b, R& c) {
    const R B0 = fma(R(3.0), d[1], -d[0]), B1 = rn_add(d[1], d[2]), B2 = fma(R(3.0), d[2], -d[3]);
    const R t0 = fma(B0, B0, E[0]), t1 = fma(B1, B1, E[1]), t2 = fma(B2, B2, E[2]);
    const R q0 = rn_mul(t0, t0), q1 = rn_mul(t1, t1), q2 = rn_mul(t2, t2);
    const R a0 = rn_mul(q1, q2), a1 = rn_mul(R(10.0), rn_mul(q0, q2)), a2 = rn_mul(q0, q1);
    const R h = rn_mul(R(0.5), rcp(rn_add(rn_add(a0, a1), a2)));
    b = rn_mul(fma(a0, B0, fma(a1, B1, rn_mul(a2, B2))), h);
    if (WANT_C) c = rn_mul(fma(a0, D2[0], fma(a1, D2[1], rn_mul(a2, D2[2]))), h);
}

// the per-position terms of zone j from w(j-2..j+2)
template <class R>
ADER_DEV void weno3_zone_terms(const R* a, R* d, R* D2, R* E) {
#pragma unroll
    for (int s = 0; s < 4; ++s) d[s] = rn_sub(a[s + 1], a[s]);
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        D2[s] = rn_sub(d[s + 1], d[s]);
        E[s] = w3_curv(D2[s]);
    }
}

template <class R>
ADER_DEV void weno3(const R* a, R& b, R& c) {
    if constexpr (sizeof(R) == 8) {
        R d[4], D2[3], E[3];
        weno3_zone_terms(a, d, D2, E);
        weno3_terms<true, R>(d, E, D2, b, c);
    } else {
        R al[3], B[3], C[3], inv;
        weno3_doubled(a, al, inv, B, C);
        const R h = R(0.5) * inv;
        b = (al[0] * B[0] + al[1] * B[1] + al[2] * B[2]) * h;
        c = (al[0] * C[0] + al[1] * C[1] + al[2] * C[2]) * h;
    }
}

// order-4 1-D WENO on the seven values a[-3..3] (a[3] = centre); returns b, c, d
template <class R>
ADER_DEV void weno4(const R* a, R& b, R& c, R& d) {
    const R um3 = a[0], um2 = a[1], um1 = a[2], u0 = a[3], up1 = a[4], up2 = a[5], up3 = a[6];
    R cb[4], cc[4], cd[4];
    // stencil {i-3..i}
    cb[0] = (R(109) * u0 - R(177) * um1 + R(87) * um2 - R(19) * um3) * R(1.0 / 60.0);
    cc[0] = (R(2) * u0 - R(5) * um1 + R(4) * um2 - um3) * R(0.5);
    cd[0] = (u0 - R(3) * um1 + R(3) * um2 - um3) * R(1.0 / 6.0);
    // stencil {i-2..i+1}
    cb[1] = (R(33) * u0 - R(63) * um1 + R(11) * um2 + R(19) * up1) * R(1.0 / 60.0);
    cc[1] = (um1 + up1 - R(2) * u0) * R(0.5);
    cd[1] = (R(3) * um1 - R(3) * u0 - um2 + up1) * R(1.0 / 6.0);
    // stencil {i-1..i+2}
    cb[2] = (R(63) * up1 - R(33) * u0 - R(19) * um1 - R(11) * up2) * R(1.0 / 60.0);
    cc[2] = (um1 + up1 - R(2) * u0) * R(0.5);
    cd[2] = (R(3) * u0 - um1 - R(3) * up1 + up2) * R(1.0 / 6.0);
    // stencil {i..i+3}
    cb[3] = (R(177) * up1 - R(109) * u0 - R(87) * up2 + R(19) * up3) * R(1.0 / 60.0);
    cc[3] = (R(2) * u0 - R(5) * up1 + R(4) * up2 - up3) * R(0.5);
    cd[3] = (R(3) * up1 - u0 - R(3) * up2 + up3) * R(1.0 / 6.0);
    const R g[4] = {R(1), R(10), R(10), R(1)};                // (1, 10, 10, 1) / 22
    R al[4], is[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const R t = cb[q] + R(0.1) * cd[q];
        is[q] = t * t + R(13.0 / 3.0) * cc[q] * cc[q] + R(781.0 / 20.0) * cd[q] * cd[q];
    }
    const R inv = weno_weights<4>(g, is, al);
    b = (al[0] * cb[0] + al[1] * cb[1] + al[2] * cb[2] + al[3] * cb[3]) * inv;
    c = (al[0] * cc[0] + al[1] * cc[1] + al[2] * cc[2] + al[3] * cc[3]) * inv;
    d = (al[0] * cd[0] + al[1] * cd[1] + al[2] * cd[2] + al[3] * cd[3]) * inv;
}

// ---------------------------------------------------------------- FP32: two stencils at once
// GB300's FP32 units execute packed pairs (one FADD2 / FMUL2 / FFMA2 does two FP32 operations), and the
// FP32 WENO kernels are bound by instruction issue, so the FP32 path blends two independent stencils
// (two variables, or two directions) per instruction: the same order-3 WENO as weno3_doubled, each
// component rounded as the scalar operations would round it, except the reciprocals (hardware
// approximations in both).
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b as b * (-1) + a: one packed FFMA2, rounded once like the subtraction (a negated operand of a
// packed addition is not folded into the instruction)
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float2 f2rcp(float2 a) { return make_float2(rcp_approx(a.x), rcp_approx(a.y)); }
__device__ __forceinline__ float2 f2s(float a) { return make_float2(a, a); }

// b (and c) of the order-3 WENO of the two stencils a[0..4].x and a[0..4].y (a[2] = centre)
template <bool WANT_C>
__device__ __forceinline__ void weno3_x2(const float2* a, float2& b, float2& c) {
    const float2 d1 = f2sub(a[1], a[0]), d2 = f2sub(a[2], a[1]), d3 = f2sub(a[3], a[2]), d4 = f2sub(a[4], a[3]);
    const float2 two = f2s(2.f);
    const float2 C0 = f2sub(d2, d1), B0 = f2fma(two, d2, C0);                  // 3 d2 - d1
    const float2 B1 = f2add(d2, d3), C1 = f2sub(d3, d2);
    const float2 C2 = f2sub(d4, d3), B2 = f2fma(two, d3, f2sub(d3, d4));      // 3 d3 - d4
    const float2 k13 = f2s(13.0f / 3.0f), eps4 = f2s((float)(4.0 * WENO_EPS));
    // q = (4 EPS + B^2 + 13/3 C^2)^2; weights (1, 10, 1) / q
    const float2 t0 = f2add(eps4, f2fma(B0, B0, f2mul(k13, f2mul(C0, C0))));
    const float2 t1 = f2add(eps4, f2fma(B1, B1, f2mul(k13, f2mul(C1, C1))));
    const float2 t2 = f2add(eps4, f2fma(B2, B2, f2mul(k13, f2mul(C2, C2))));
    const float2 a0 = f2rcp(f2mul(t0, t0));
    const float2 a1 = f2mul(f2s(10.f), f2rcp(f2mul(t1, t1)));
    const float2 a2 = f2rcp(f2mul(t2, t2));
    const float2 h = f2mul(f2s(0.5f), f2rcp(f2add(f2add(a0, a1), a2)));
    b = f2mul(f2fma(a0, B0, f2fma(a1, B1, f2mul(a2, B2))), h);
    if (WANT_C) c = f2mul(f2fma(a0, C0, f2fma(a1, C1, f2mul(a2, C2))), h);
}

template <class R>
ADER_DEV R slope(const R* a) {
    R b, c;
    if constexpr (sizeof(R) == 8) {     // the slope alone: no curvature blend
        R d[4], D2[3], E[3];
        weno3_zone_terms(a, d, D2, E);
        weno3_terms<false, R>(d, E, D2, b, c);
    } else {
        weno3(a, b, c);
    }
    return b;
}



// slope along direction d of the field F at zone (i, j, k)
template <class R>
ADER_DEV R slope_of(const Grid& g, const R* __restrict__ F, int i, int j, int k, int d) {
    R a[5];
#pragma unroll
    for (int o = -2; o <= 2; ++o) {
        const long long z = ((long long)k * g.ny + j) * g.nx + i;
        a[o + 2] = F[o == 0 ? z : nbr_along(g, z, i, j, k, d, o)];
    }
    return slope(a);
}


// ---------------------------------------------------------------- per-zone bodies of the kernels
// 1-D moments of zone z (S1 layout in recon.cu).  Variables 0..4 are read
// from U; for MHD (NV = 8) variable 5 + e is the zone field B_e read from ZB,
// whose moments along e come from the face-B WENO (zone_face_b), so only the
// two transverse directions are reconstructed here.
// T: the type U is read in (double, or the FP32 copy of FP32-bulk steps).
template <int ORDER, int NV, class R, class T>
ADER_DEV void zone_weno1d(const Grid& g, const T* __restrict__ U, const R* __restrict__ ZB,
                          R* __restrict__ S1, long long z) {
    int i, j, k;
    zone_ijk(g, z, i, j, k);
#ifdef __CUDA_ARCH__
    if constexpr (ORDER <= 3 && NV == 5 && sizeof(R) == 4 && sizeof(T) == 4) {
        // FP32 Euler: the fifteen stencils (variable v, direction d) in seven pairs and one single
        long long off[3][4];
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
            for (int o = 0; o < 4; ++o) off[d][o] = nbr_along(g, z, i, j, k, d, o < 2 ? o - 2 : o - 1) - z;
        float st[15][5];
#pragma unroll
        for (int q = 0; q < 15; ++q) {
            const int v = q / 3, d = q % 3;
            const T* Uv = U + (long long)v * g.n + z;
            st[q][0] = Uv[off[d][0]];
            st[q][1] = Uv[off[d][1]];
            st[q][2] = Uv[0];
            st[q][3] = Uv[off[d][2]];
            st[q][4] = Uv[off[d][3]];
        }
#pragma unroll
        for (int q = 0; q < 15; q += 2) {
            float2 a[5], b, c;
            if (q + 1 < 15) {
#pragma unroll
                for (int o = 0; o < 5; ++o) a[o] = make_float2(st[q][o], st[q + 1][o]);
            } else {
#pragma unroll
                for (int o = 0; o < 5; ++o) a[o] = make_float2(st[q][o], st[q][o]);
            }
            weno3_x2<ORDER == 3>(a, b, c);
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                if (q + u >= 15) break;
                const int v = (q + u) / 3, d = (q + u) % 3;
                S1[((0 * 3 + d) * NV + v) * g.n + z] = u ? b.y : b.x;
                if (ORDER == 3) S1[((1 * 3 + d) * NV + v) * g.n + z] = u ? c.y : c.x;
            }
        }
    } else
#endif
    {
        constexpr int RAD = ORDER == 4 ? 3 : 2;
        // the stencil's neighbour offsets, once for all variables (offset 0 is the zone itself)
        long long off[3][2 * RAD + 1];
    #pragma unroll
        for (int d = 0; d < 3; ++d)
    #pragma unroll
            for (int o = -RAD; o <= RAD; ++o) off[d][o + RAD] = o == 0 ? 0 : nbr_along(g, z, i, j, k, d, o) - z;
        // per variable the three directions' moments before any store (a store could alias the next
        // loads for all the compiler knows, and would hold them back)
        for (int v = 0; v < NV; ++v) {
            const T* Uv = v < 5 ? U + (long long)v * g.n + z : nullptr;
            const R* Bv = v >= 5 ? ZB + (long long)(v - 5) * g.n + z : nullptr;
            const R centre = v < 5 ? R(Uv[0]) : Bv[0];
            R m[3][3];
    #pragma unroll
            for (int d = 0; d < 3; ++d) {
                if (v >= 5 && d == v - 5) continue;
                R a[2 * RAD + 1];
    #pragma unroll
                for (int o = -RAD; o <= RAD; ++o) {
                    if (o == 0)
                        a[RAD] = centre;
                    else
                        a[o + RAD] = v < 5 ? R(Uv[off[d][o + RAD]]) : Bv[off[d][o + RAD]];
                }
                if (ORDER == 4)
                    weno4(a, m[d][0], m[d][1], m[d][2]);
                else if (ORDER == 3)
                    weno3(a, m[d][0], m[d][1]);
                else
                    m[d][0] = slope(a);
            }
    #pragma unroll
            for (int d = 0; d < 3; ++d) {
                if (v >= 5 && d == v - 5) continue;
                S1[((0 * 3 + d) * NV + v) * g.n + z] = m[d][0];
                if (ORDER >= 3) S1[((1 * 3 + d) * NV + v) * g.n + z] = m[d][1];
                if (ORDER == 4) S1[((2 * 3 + d) * NV + v) * g.n + z] = m[d][2];
            }
        }
    }
}

// first-level cross moments w8 w9 w10 (w14..w19 at order 4) of zone z
template <int ORDER, int NV, class R>
ADER_DEV void zone_cross1(const Grid& g, const R* __restrict__ S1, R* __restrict__ S2, long long z) {
    int i, j, k;
    zone_ijk(g, z, i, j, k);
#ifdef __CUDA_ARCH__
    if constexpr (sizeof(R) == 4) {
        // FP32: the two slopes of each first-level cross moment as one packed pair (weno3_x2); the
        // neighbour offsets once per zone
        long long off[3][5];
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
            for (int o = 0; o < 5; ++o) off[d][o] = o == 2 ? 0 : nbr_along(g, z, i, j, k, d, o - 2) - z;
        // per variable every result before any store: a store could alias the next loads for all the
        // compiler knows (the batched kernels pass no restricted pointers), and would hold them back
        for (int v = 0; v < NV; ++v) {
            const R* w2 = S1 + ((0 * 3 + 0) * NV + v) * g.n + z;
            const R* w3 = S1 + ((0 * 3 + 1) * NV + v) * g.n + z;
            const R* w4 = S1 + ((0 * 3 + 2) * NV + v) * g.n + z;
            float2 a[5], r[6], unused;
#pragma unroll
            for (int o = 0; o < 5; ++o) a[o] = make_float2(w2[off[1][o]], w3[off[0][o]]);
            weno3_x2<false>(a, r[0], unused);
#pragma unroll
            for (int o = 0; o < 5; ++o) a[o] = make_float2(w3[off[2][o]], w4[off[1][o]]);
            weno3_x2<false>(a, r[1], unused);
#pragma unroll
            for (int o = 0; o < 5; ++o) a[o] = make_float2(w2[off[2][o]], w4[off[0][o]]);
            weno3_x2<false>(a, r[2], unused);
            if (ORDER == 4) {
                const R* w5 = S1 + ((1 * 3 + 0) * NV + v) * g.n + z;
                const R* w6 = S1 + ((1 * 3 + 1) * NV + v) * g.n + z;
                const R* w7 = S1 + ((1 * 3 + 2) * NV + v) * g.n + z;
                const R* src[6] = {w5, w5, w6, w6, w7, w7};
                const int dir[6] = {1, 2, 0, 2, 0, 1};             // w14 .. w19
#pragma unroll
                for (int c = 0; c < 6; c += 2) {
#pragma unroll
                    for (int o = 0; o < 5; ++o) a[o] = make_float2(src[c][off[dir[c]][o]], src[c + 1][off[dir[c + 1]][o]]);
                    weno3_x2<false>(a, r[3 + c / 2], unused);
                }
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) S2[(c * NV + v) * g.n + z] = 0.5f * (r[c].x + r[c].y);
            if (ORDER == 4) {
#pragma unroll
                for (int c = 0; c < 6; c += 2) {
                    S2[((3 + c) * NV + v) * g.n + z] = r[3 + c / 2].x;
                    S2[((4 + c) * NV + v) * g.n + z] = r[3 + c / 2].y;
                }
            }
        }
    } else
#endif
    for (int v = 0; v < NV; ++v) {
        const R* w2 = S1 + ((0 * 3 + 0) * NV + v) * g.n;
        const R* w3 = S1 + ((0 * 3 + 1) * NV + v) * g.n;
        const R* w4 = S1 + ((0 * 3 + 2) * NV + v) * g.n;
        S2[(0 * NV + v) * g.n + z] = R(0.5) * (slope_of(g, w2, i, j, k, 1) + slope_of(g, w3, i, j, k, 0));
        S2[(1 * NV + v) * g.n + z] = R(0.5) * (slope_of(g, w3, i, j, k, 2) + slope_of(g, w4, i, j, k, 1));
        S2[(2 * NV + v) * g.n + z] = R(0.5) * (slope_of(g, w2, i, j, k, 2) + slope_of(g, w4, i, j, k, 0));
        if (ORDER == 4) {
            const R* w5 = S1 + ((1 * 3 + 0) * NV + v) * g.n;
            const R* w6 = S1 + ((1 * 3 + 1) * NV + v) * g.n;
            const R* w7 = S1 + ((1 * 3 + 2) * NV + v) * g.n;
            S2[(3 * NV + v) * g.n + z] = slope_of(g, w5, i, j, k, 1);   // w14
            S2[(4 * NV + v) * g.n + z] = slope_of(g, w5, i, j, k, 2);   // w15
            S2[(5 * NV + v) * g.n + z] = slope_of(g, w6, i, j, k, 0);   // w16
            S2[(6 * NV + v) * g.n + z] = slope_of(g, w6, i, j, k, 2);   // w17
            S2[(7 * NV + v) * g.n + z] = slope_of(g, w7, i, j, k, 0);   // w18
            S2[(8 * NV + v) * g.n + z] = slope_of(g, w7, i, j, k, 1);   // w19
        }
    }
}

// w20 of zone z from the first-level cross moments of its neighbours
template <int NV, class R>
ADER_DEV void zone_cross2(const Grid& g, R* __restrict__ S2, long long z) {
    int i, j, k;
    zone_ijk(g, z, i, j, k);
    for (int v = 0; v < NV; ++v) {
        const R* w8 = S2 + (0 * NV + v) * g.n;
        const R* w9 = S2 + (1 * NV + v) * g.n;
        const R* w10 = S2 + (2 * NV + v) * g.n;
        S2[(9 * NV + v) * g.n + z] = (slope_of(g, w8, i, j, k, 2) + slope_of(g, w9, i, j, k, 0) +
                                      slope_of(g, w10, i, j, k, 1)) * R(1.0 / 3.0);
    }
}

// ---------------------------------------------------------------- Sec. III: zone B from face B
// Face-B WENO along direction e for zone z: the zone-averaged normal field b0
// (written to ZB[e]) and its normal moments b_x, b_xx, b_xxx (written to the
// S1 slots of variable 5 + e, direction e).  Bf[e][zone i] is B_e on face i - 1/2.
// Order 2: mean and difference (Sec. III, opening).  Order 3: Eqs. 21-24 with
// linear weights (1/2, 1/2).  Order 4: Eqs. 25-29 with (1/4, 1/2, 1/4).
template <int ORDER, class R>
ADER_DEV void zone_face_b(const Grid& g, const double* __restrict__ Bf, R* __restrict__ ZB, R* __restrict__ S1,
                          long long z) {
    int i, j, k;
    zone_ijk(g, z, i, j, k);
    constexpr int NV = 8;
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        const double* B = Bf + (long long)e * g.n;
        auto at = [&](int o) { return R(B[nbr_along(g, z, i, j, k, e, o)]); };
        const R Bm = at(0), Bp = at(1);                   // faces i - 1/2 and i + 1/2
        R m[4];
        if (ORDER == 2) {
            m[0] = R(0.5) * (Bp + Bm);
            m[1] = Bp - Bm;
        } else if (ORDER == 3) {
            const R Bmm = at(-1), Bpp = at(2);
            const R s1[3] = {(R(8) * Bm - Bmm + R(5) * Bp) * R(1.0 / 12.0), Bp - Bm, (Bp + Bmm - R(2) * Bm) * R(0.5)};
            const R s2[3] = {(R(8) * Bp - Bpp + R(5) * Bm) * R(1.0 / 12.0), Bp - Bm, (Bm + Bpp - R(2) * Bp) * R(0.5)};
            const R k13 = R(13.0 / 3.0);
            const R g[2] = {R(1), R(1)};                      // (1/2, 1/2)
            const R is[2] = {s1[1] * s1[1] + k13 * s1[2] * s1[2], s2[1] * s2[1] + k13 * s2[2] * s2[2]};
            R al[2];
            const R inv = weno_weights<2>(g, is, al);
#pragma unroll
            for (int r = 0; r < 3; ++r) m[r] = (al[0] * s1[r] + al[1] * s2[r]) * inv;
        } else {
            const R Bmm = at(-1), Bmmm = at(-2), Bpp = at(2), Bppp = at(3);
            const R c[3][4] = {
                {(R(9) * Bp + R(19) * Bm - R(5) * Bmm + Bmmm) * R(1.0 / 24.0),
                 (R(59) * Bp - R(57) * Bm - R(3) * Bmm + Bmmm) * R(1.0 / 60.0),
                 (R(3) * Bp - R(7) * Bm + R(5) * Bmm - Bmmm) * R(0.25),
                 (Bp - R(3) * Bm + R(3) * Bmm - Bmmm) * R(1.0 / 6.0)},                       // Eq. 26
                {(-Bpp + R(13) * Bp + R(13) * Bm - Bmm) * R(1.0 / 24.0),
                 (-Bpp + R(63) * Bp - R(63) * Bm + Bmm) * R(1.0 / 60.0),
                 (Bpp - Bp - Bm + Bmm) * R(0.25),
                 (Bpp - R(3) * Bp + R(3) * Bm - Bmm) * R(1.0 / 6.0)},                        // Eq. 27
                {(Bppp - R(5) * Bpp + R(19) * Bp + R(9) * Bm) * R(1.0 / 24.0),
                 (-Bppp + R(3) * Bpp + R(57) * Bp - R(59) * Bm) * R(1.0 / 60.0),
                 (-Bppp + R(5) * Bpp - R(7) * Bp + R(3) * Bm) * R(0.25),
                 (Bppp - R(3) * Bpp + R(3) * Bp - Bm) * R(1.0 / 6.0)}};                      // Eq. 28
            const R gl[3] = {R(1), R(2), R(1)};               // (1/4, 1/2, 1/4)
            R al[3], is[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const R t = c[q][1] + R(0.1) * c[q][3];
                is[q] = t * t + R(13.0 / 3.0) * c[q][2] * c[q][2] + R(781.0 / 20.0) * c[q][3] * c[q][3];
            }
            const R inv = weno_weights<3>(gl, is, al);
#pragma unroll
            for (int r = 0; r < 4; ++r) m[r] = (al[0] * c[0][r] + al[1] * c[1][r] + al[2] * c[2][r]) * inv;
        }
        ZB[(long long)e * g.n + z] = m[0];
#pragma unroll
        for (int r = 0; r < ORDER - 1; ++r) S1[((r * 3 + e) * NV + 5 + e) * g.n + z] = m[r + 1];
    }
}

}  // namespace ader
