// Learned initial guess of the third-order ADER-CG predictor.
//
// A small MLP (in -> 128 -> 128 -> out, GELU) maps a zone's normalised
// spatial modes to its evolutionary modes u11..u15, which then start the
// Picard iteration instead of zeros; the converged iteration stays the reference
// for the result.  The normalisation makes the map dimensionless and exact for
// uniform zones:
//   scales   s_rho = w1(rho), s_E = w1(eps), c = sqrt(s_E / s_rho),
//            s_m = s_rho c (momentum), s_B = sqrt(8 pi s_E) (field);
//   slopes   r = w2..w10 of every variable over its scale; their magnitude
//            g = max |r|;
//   features r / g; the zone means of momentum (and field) over their scales;
//            the Courant numbers c dt/dx, c dt/dy, c dt/dz; and g;
//   targets  u11..u15 of each variable over (its scale x sigma x g),
//            sigma = c (dt/dx + dt/dy + dt/dz).
// A zone with g <= GUESS_MAG_MIN (uniform to round-off, at rest or moving)
// has no time evolution to speak of: its guess is zero and it is not a
// training sample.  The threshold is a round-off level: with fused
// multiply-adds the stencil differences of uniform data leave residuals near
// 1e-16.
// Parameters are packed FP32: W1 (H x IN, row-major), b1 (H), W2 (H x H),
// b2 (H), W3 (OUT x H), b3 (OUT).
#pragma once
#include <math.h>

#include "common.cuh"

namespace ader {

constexpr int MLP_HIDDEN = 128;
constexpr double GUESS_MAG_MIN = 1e-12;

ADER_DEV constexpr int mlp_in(int nv) { return nv == 8 ? 82 : 52; }
ADER_DEV constexpr int mlp_out(int nv) { return 5 * nv; }
ADER_DEV constexpr long long mlp_params(int nv) {
    return (long long)MLP_HIDDEN * mlp_in(nv) + MLP_HIDDEN + (long long)MLP_HIDDEN * MLP_HIDDEN + MLP_HIDDEN +
           (long long)mlp_out(nv) * MLP_HIDDEN + mlp_out(nv);
}

// tanh form of GELU
ADER_DEV float gelu(float x) {
    const float t = tanhf(0.7978845608028654f * (x + 0.044715f * x * x * x));
    return 0.5f * x * (1.0f + t);
}

ADER_DEV float gelu_grad(float x) {
    const float k = 0.7978845608028654f;
    const float u = k * (x + 0.044715f * x * x * x);
    const float t = tanhf(u);
    return 0.5f * (1.0f + t) + 0.5f * x * (1.0f - t * t) * k * (1.0f + 3.0f * 0.044715f * x * x);
}

template <int NV, class R>
struct GuessScales {
    double s[NV];
    double sigma;
    bool ok;
};

template <int NV, class R>
ADER_DEV GuessScales<NV, R> guess_scales(const Vec<NV, R>* m, double cx, double cy, double cz) {
    GuessScales<NV, R> g;
    const double rho = (double)m[1][0], E = (double)m[1][4];
    g.ok = rho > 0.0 && E > 0.0;
    const double c = g.ok ? sqrt(E / rho) : 1.0;
    g.s[0] = rho;
    g.s[1] = g.s[2] = g.s[3] = rho * c;
    g.s[4] = E;
    if constexpr (NV == 8) g.s[5] = g.s[6] = g.s[7] = sqrt(8.0 * 3.14159265358979323846 * E);
    g.sigma = c * (cx + cy + cz);
    g.ok = g.ok && g.sigma > 0.0;
    return g;
}

// features of a zone (order 3) into x[mlp_in(NV)]; returns the slope magnitude g
template <int NV, class R>
ADER_DEV double guess_features(const Vec<NV, R>* m, const GuessScales<NV, R>& g, double cx, double cy, double cz,
                               float* x) {
    double r[9 * NV];
    double mag = 0.0;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const double inv = 1.0 / g.s[v];
#pragma unroll
        for (int k = 2; k <= 10; ++k) {
            r[v * 9 + k - 2] = (double)m[k][v] * inv;
            mag = fmax(mag, fabs(r[v * 9 + k - 2]));
        }
    }
    const double im = mag > 0.0 ? 1.0 / mag : 0.0;
#pragma unroll
    for (int q = 0; q < 9 * NV; ++q) x[q] = (float)(r[q] * im);
    int n = 9 * NV;
#pragma unroll
    for (int v = 1; v < NV; ++v)
        if (v != 4) x[n++] = (float)((double)m[1][v] / g.s[v]);     // Mach (and field) numbers
    const double c = g.sigma / (cx + cy + cz);
    x[n++] = (float)(c * cx);
    x[n++] = (float)(c * cy);
    x[n++] = (float)(c * cz);
    x[n] = (float)mag;
    return mag;
}

// g of guess_features_f32 alone (the same FP32 arithmetic): the slope magnitude that decides whether a
// zone runs the network; 0 where the scales are not positive.
template <int NV, class R>
ADER_DEV float guess_mag_f32(const Vec<NV, R>* m) {
    const float rho = (float)m[1][0], E = (float)m[1][4];
    if (!(rho > 0.f) || !(E > 0.f)) return 0.f;
    const float c = sqrtf(E / rho);
    float s[NV];
    s[0] = rho;
    s[1] = s[2] = s[3] = rho * c;
    s[4] = E;
    if constexpr (NV == 8) s[5] = s[6] = s[7] = sqrtf(8.0f * 3.14159265358979f * E);
    float mag = 0.f;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const float inv = 1.0f / s[v];
#pragma unroll
        for (int k = 2; k <= 10; ++k) mag = fmaxf(mag, fabsf((float)m[k][v] * inv));
    }
    return mag;
}

// The same features in FP32 arithmetic (inference: they feed FP16 operands),
// plus the output scale of each variable, s_v sigma g, in sv.  Returns g, or
// 0 where the scales are not positive.
template <int NV, class R>
ADER_DEV float guess_features_f32(const Vec<NV, R>* m, float cx, float cy, float cz, float* x, float* sv) {
    const float rho = (float)m[1][0], E = (float)m[1][4];
    if (!(rho > 0.f) || !(E > 0.f)) return 0.f;
    const float c = sqrtf(E / rho);
    float s[NV];
    s[0] = rho;
    s[1] = s[2] = s[3] = rho * c;
    s[4] = E;
    if constexpr (NV == 8) s[5] = s[6] = s[7] = sqrtf(8.0f * 3.14159265358979f * E);
    float inv[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) inv[v] = 1.0f / s[v];
    float mag = 0.f;
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
        for (int k = 2; k <= 10; ++k) {
            x[v * 9 + k - 2] = (float)m[k][v] * inv[v];
            mag = fmaxf(mag, fabsf(x[v * 9 + k - 2]));
        }
    const float im = mag > 0.f ? 1.0f / mag : 0.f;
#pragma unroll
    for (int q = 0; q < 9 * NV; ++q) x[q] *= im;
    int n = 9 * NV;
#pragma unroll
    for (int v = 1; v < NV; ++v)
        if (v != 4) x[n++] = (float)m[1][v] * inv[v];
    x[n++] = c * cx;
    x[n++] = c * cy;
    x[n++] = c * cz;
    x[n] = mag;
    const float sigma = c * (cx + cy + cz);
#pragma unroll
    for (int v = 0; v < NV; ++v) sv[v] = s[v] * sigma * mag;
    return mag;
}

// normalised targets of a zone: t[j*NV + v] = u_{11+j}[v] / (s_v sigma g)
template <int NV, class R>
ADER_DEV void guess_targets(const Vec<NV, R>* m, const GuessScales<NV, R>& g, double mag, float* t) {
#pragma unroll
    for (int j = 0; j < 5; ++j)
#pragma unroll
        for (int v = 0; v < NV; ++v) t[j * NV + v] = (float)((double)m[11 + j][v] / (g.s[v] * g.sigma * mag));
}

}  // namespace ader
