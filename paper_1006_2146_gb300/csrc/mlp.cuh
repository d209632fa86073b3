// Learned initial guess of the third-order ADER-CG predictor.
//
// A small MLP (in -> 128 -> 128 -> out, GELU) maps a zone's normalised
// spatial modes to its evolutionary modes u11..u15, which then start the
// Picard iteration instead of zeros; the converged iteration stays the judge
// of the result.  The normalisation makes the map dimensionless:
//   scales   s_rho = w1(rho), s_E = w1(eps), c = sqrt(s_E / s_rho),
//            s_m = s_rho c (momentum), s_B = sqrt(8 pi s_E) (field);
//   features w2..w10 of rho and eps, w1..w10 of each momentum (and field)
//            component, each over its scale, and the Courant numbers
//            c dt/dx, c dt/dy, c dt/dz;
//   targets  u11..u15 of each variable over (its scale x sigma),
//            sigma = c (dt/dx + dt/dy + dt/dz).
// Parameters are packed FP32: W1 (H x IN, row-major), b1 (H), W2 (H x H),
// b2 (H), W3 (OUT x H), b3 (OUT).
#pragma once
#include <math.h>

#include "common.cuh"

namespace ader {

constexpr int MLP_HIDDEN = 128;

ADER_DEV constexpr int mlp_in(int nv) { return nv == 8 ? 81 : 51; }
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

// features of a zone (order 3) into x[mlp_in(NV)]
template <int NV, class R>
ADER_DEV void guess_features(const Vec<NV, R>* m, const GuessScales<NV, R>& g, double cx, double cy, double cz,
                             float* x) {
    int n = 0;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const double inv = 1.0 / g.s[v];
        const int k0 = (v == 0 || v == 4) ? 2 : 1;
#pragma unroll
        for (int k = k0; k <= 10; ++k) x[n++] = (float)((double)m[k][v] * inv);
    }
    const double c = g.sigma / (cx + cy + cz);
    x[n++] = (float)(c * cx);
    x[n++] = (float)(c * cy);
    x[n++] = (float)(c * cz);
}

// normalised targets of a zone: t[j*NV + v] = u_{11+j}[v] / (s_v sigma)
template <int NV, class R>
ADER_DEV void guess_targets(const Vec<NV, R>* m, const GuessScales<NV, R>& g, float* t) {
#pragma unroll
    for (int j = 0; j < 5; ++j)
#pragma unroll
        for (int v = 0; v < NV; ++v) t[j * NV + v] = (float)((double)m[11 + j][v] / (g.s[v] * g.sigma));
}

// One zone's MLP evaluation, FP32.  Layer 2 is evaluated in chunks of 8
// outputs that are immediately folded into layer 3, so only the first hidden
// layer is held whole.
template <int IN, int OUT>
ADER_DEV void mlp_eval(const float* __restrict__ P, const float* x, float* y) {
    constexpr int H = MLP_HIDDEN;
    const float* W1 = P;
    const float* b1 = W1 + H * IN;
    const float* W2 = b1 + H;
    const float* b2 = W2 + H * H;
    const float* W3 = b2 + H;
    const float* b3 = W3 + OUT * H;
    float h1[H];
#pragma unroll 4
    for (int i = 0; i < H; ++i) {
        float s = b1[i];
#pragma unroll
        for (int k = 0; k < IN; ++k) s = fmaf(W1[i * IN + k], x[k], s);
        h1[i] = gelu(s);
    }
#pragma unroll
    for (int o = 0; o < OUT; ++o) y[o] = b3[o];
    for (int c = 0; c < H; c += 8) {
        float h2[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            float s = b2[c + r];
#pragma unroll 16
            for (int k = 0; k < H; ++k) s = fmaf(W2[(c + r) * H + k], h1[k], s);
            h2[r] = gelu(s);
        }
#pragma unroll
        for (int o = 0; o < OUT; ++o)
#pragma unroll
            for (int r = 0; r < 8; ++r) y[o] = fmaf(W3[o * H + c + r], h2[r], y[o]);
    }
}

// Replace the evolutionary modes m[11..15] by the MLP's guess (order 3).
template <int NV, class R>
ADER_DEV void learned_guess(const float* __restrict__ P, Vec<NV, R>* m, R gamma, R cx, R cy, R cz) {
    (void)gamma;
    const GuessScales<NV, R> g = guess_scales<NV, R>(m, (double)cx, (double)cy, (double)cz);
    if (!g.ok) return;
    float x[mlp_in(NV)], y[mlp_out(NV)];
    guess_features<NV, R>(m, g, (double)cx, (double)cy, (double)cz, x);
    mlp_eval<mlp_in(NV), mlp_out(NV)>(P, x, y);
#pragma unroll
    for (int j = 0; j < 5; ++j)
#pragma unroll
        for (int v = 0; v < NV; ++v) m[11 + j][v] = R((double)y[j * NV + v] * g.s[v] * g.sigma);
}

}  // namespace ader
