// Third order: ADER-CG predictor (modal Sec. IV.2, nodal App. B) and the
// x+ face quantities (Sec. V.2, App. D) of one zone.
//
// Modes m[1..15] use the paper's numbering (Eq. 15): m[1..10] = w1..w10,
// m[11..15] = u11..u15.  The scaled fluxes of Eq. 5 are c_d * F_d with
// c_d = dt / dx_d; the extraction rules are linear, so the scaling is applied
// to the extracted flux modes.
#pragma once
#include "common.cuh"
#include "modes.cuh"

namespace ader {
namespace o3 {


// ------------------------------------------------------------------ modal, Sec. IV.2
// SRC: with a non-stiff source (s = dt S at every node of the current iterate,
// Eqs. 40-43 with f, g, h -> s, Eq. 36 with its source terms); sdt receives
// dt S-bar of Eq. 44 from the source at the final iterate.
template <int NV, class R, bool SRC = false>
ADER_DEV void predict_modal(Vec<NV, R>* m, R gm1, R cx, R cy, R cz, PredCtl& ctl, const Src<R>* src = nullptr,
                            Vec<NV, R>* sdt = nullptr) {
    // Eq. 38: the thirteen tau = 0 nodes of Eq. 37
    Vec<NV, R> u[14];
    u[1] = m[1] - (m[5] + m[6] + m[7]) / 12.0;
    u[2] = u[1] + 0.5 * (m[2] + m[3]) + 0.25 * (m[5] + m[6] + m[8]);
    u[3] = u[2] - m[3] - 0.5 * m[8];
    u[4] = u[1] + 0.5 * (m[2] + m[4]) + 0.25 * (m[5] + m[7] + m[10]);
    u[5] = u[4] - m[4] - 0.5 * m[10];
    u[6] = u[3] - m[2] + m[3];
    u[7] = u[2] - m[2] - m[3];
    u[8] = u[5] - m[2] + m[4];
    u[9] = u[4] - m[2] - m[4];
    u[10] = u[1] + 0.5 * (m[3] + m[4]) + 0.25 * (m[6] + m[7] + m[9]);
    u[11] = u[10] - m[3] - 0.5 * m[9];
    u[12] = u[11] + m[3] - m[4];
    u[13] = u[10] - m[3] - m[4];
    // fluxes at the tau = 0 nodes, built once (Sec. IV.2)
    Vec<NV, R> f[14], g[14], h[14];
#pragma unroll
    for (int n = 1; n <= 13; ++n) {
        const Prim<NV, R> q = primitives(u[n], gm1);
        f[n] = flux_from<0>(u[n], q);
        g[n] = flux_from<1>(u[n], q);
        h[n] = flux_from<2>(u[n], q);
    }
    // Eqs. 40-42, tau = 0 modes
    const Vec<NV, R> q1 = f[2] + f[3] + f[4] + f[5], q2 = f[6] + f[7] + f[8] + f[9], q3 = f[10] + f[11] + f[12] + f[13];
    const Vec<NV, R> F2 = scale(cx, 0.25 * (q1 - q2));
    const Vec<NV, R> F5 = scale(cx, 0.5 * (q1 + q2 - q3) - 2.0 * f[1]);
    const Vec<NV, R> F8 = scale(cx, f[2] - f[3] - f[6] + f[7]);
    const Vec<NV, R> F10 = scale(cx, f[4] - f[5] - f[8] + f[9]);
    const Vec<NV, R> q4 = g[2] + g[6] + g[10] + g[12], q5 = g[3] + g[7] + g[11] + g[13], q6 = g[4] + g[5] + g[8] + g[9];
    const Vec<NV, R> G3 = scale(cy, 0.25 * (q4 - q5));
    const Vec<NV, R> G6 = scale(cy, 0.5 * (q4 + q5 - q6) - 2.0 * g[1]);
    const Vec<NV, R> G8 = scale(cy, g[2] - g[3] - g[6] + g[7]);
    const Vec<NV, R> G9 = scale(cy, g[10] - g[11] - g[12] + g[13]);
    const Vec<NV, R> q7 = h[4] + h[8] + h[10] + h[11], q8 = h[5] + h[9] + h[12] + h[13], q9 = h[2] + h[3] + h[6] + h[7];
    const Vec<NV, R> H4 = scale(cz, 0.25 * (q7 - q8));
    const Vec<NV, R> H7 = scale(cz, 0.5 * (q7 + q8 - q9) - 2.0 * h[1]);
    const Vec<NV, R> H9 = scale(cz, h[10] - h[11] - h[12] + h[13]);
    const Vec<NV, R> H10 = scale(cz, h[4] - h[5] - h[8] + h[9]);
    // source modes from the tau = 0 nodes (Eqs. 40-43 with f, g, h -> s), built once
    Vec<NV, R> S1, S2, S3, S4, s1;
    if constexpr (SRC) {
        Vec<NV, R> sn[14];
#pragma unroll
        for (int n = 1; n <= 13; ++n) sn[n] = source_at(u[n], *src);
        const Vec<NV, R> a1 = sn[2] + sn[3] + sn[4] + sn[5], a2 = sn[6] + sn[7] + sn[8] + sn[9];
        const Vec<NV, R> a3 = sn[10] + sn[11] + sn[12] + sn[13];
        const Vec<NV, R> b4 = sn[2] + sn[6] + sn[10] + sn[12], b5 = sn[3] + sn[7] + sn[11] + sn[13];
        const Vec<NV, R> b6 = sn[4] + sn[5] + sn[8] + sn[9];
        const Vec<NV, R> c7 = sn[4] + sn[8] + sn[10] + sn[11], c8 = sn[5] + sn[9] + sn[12] + sn[13];
        const Vec<NV, R> c9 = sn[2] + sn[3] + sn[6] + sn[7];
        S2 = 0.25 * (a1 - a2);
        S3 = 0.25 * (b4 - b5);
        S4 = 0.25 * (c7 - c8);
        const Vec<NV, R> S5 = 0.5 * (a1 + a2 - a3) - 2.0 * sn[1];
        const Vec<NV, R> S6 = 0.5 * (b4 + b5 - b6) - 2.0 * sn[1];
        const Vec<NV, R> S7 = 0.5 * (c7 + c8 - c9) - 2.0 * sn[1];
        s1 = sn[1];
        S1 = s1 + (S5 + S6 + S7) / 12.0;
    }
    const bool conv = positive_arg(ctl.tol);
    const int cap = conv ? ctl.max_iter : ctl.n_iter;
    const R ref = max_abs(m[1]) + R(sizeof(R) == 8 ? 1e-300 : 1e-30);   // never zero in R
    ctl.iters = 0;
    ctl.capped = conv;
    for (int it = 0; it < cap; ++it) {
        // Eq. 39: the tau = 1/2 nodes (node 20 serves only source terms)
        const Vec<NV, R> u14 = 0.25 * (u[2] + u[3] + u[4] + u[5] + m[12] + m[13]) + 0.5 * m[11] - 0.125 * (m[6] + m[7]);
        const Vec<NV, R> u16 = 0.25 * (u[2] + u[6] + u[10] + u[12] + m[12] + m[14]) + 0.5 * m[11] - 0.125 * (m[5] + m[7]);
        const Vec<NV, R> u18 = 0.25 * (u[4] + u[8] + u[10] + u[11] + m[12] + m[15]) + 0.5 * m[11] - 0.125 * (m[5] + m[6]);
        const Vec<NV, R> u15 = u14 - m[2] - 0.5 * m[13];
        const Vec<NV, R> u17 = u16 - m[3] - 0.5 * m[14];
        const Vec<NV, R> u19 = u18 - m[4] - 0.5 * m[15];
        // time modes of Eqs. 40-42
        const Vec<NV, R> F13 = 2.0 * (scale(cx, flux<0>(u14, gm1) - flux<0>(u15, gm1)) - F2);
        const Vec<NV, R> G14 = 2.0 * (scale(cy, flux<1>(u16, gm1) - flux<1>(u17, gm1)) - G3);
        const Vec<NV, R> H15 = 2.0 * (scale(cz, flux<2>(u18, gm1) - flux<2>(u19, gm1)) - H4);
        // Eq. 36
        Vec<NV, R> n11 = -(F2 + G3 + H4);
        Vec<NV, R> n12 = -0.5 * (F13 + G14 + H15);
        Vec<NV, R> n13 = -(2.0 * F5 + G8 + H10);
        Vec<NV, R> n14 = -(F8 + 2.0 * G6 + H9);
        Vec<NV, R> n15 = -(F10 + G9 + 2.0 * H7);
        if constexpr (SRC) {
            const Vec<NV, R> s14 = source_at(u14, *src), s15 = source_at(u15, *src);
            const Vec<NV, R> s16 = source_at(u16, *src), s17 = source_at(u17, *src);
            const Vec<NV, R> s18 = source_at(u18, *src), s19 = source_at(u19, *src);
            const Vec<NV, R> s20 = source_at(u[1] + m[11] + m[12], *src);
            const Vec<NV, R> S13 = 2.0 * (s14 - s15 - S2), S14 = 2.0 * (s16 - s17 - S3), S15 = 2.0 * (s18 - s19 - S4);
            const Vec<NV, R> S11 = 2.0 * (s14 + s15 + s16 + s17 + s18 + s19 - 6.0 * S1) / 3.0 - s20 + s1;
            const Vec<NV, R> S12 = s20 - s1 - S11;
            n11 += S1 - 0.3 * S12;
            n12 += 0.5 * S11 + 0.6 * S12;
            n13 += S2 + (2.0 / 3.0) * S13;
            n14 += S3 + (2.0 / 3.0) * S14;
            n15 += S4 + (2.0 / 3.0) * S15;
        }
        R change = R(0);
        if (conv)
            change = fmax(fmax(fmax(max_abs_diff(n11, m[11]), max_abs_diff(n12, m[12])),
                               fmax(max_abs_diff(n13, m[13]), max_abs_diff(n14, m[14]))),
                          max_abs_diff(n15, m[15]));
        m[11] = n11;
        m[12] = n12;
        m[13] = n13;
        m[14] = n14;
        m[15] = n15;
        ++ctl.iters;
        if (conv && change < R(ctl.tol) * ref) {
            ctl.capped = false;
            break;
        }
    }
    if constexpr (SRC) {        // Eq. 44 from the source at the final iterate's tau > 0 nodes (Eq. 39)
        const Vec<NV, R> u14 = 0.25 * (u[2] + u[3] + u[4] + u[5] + m[12] + m[13]) + 0.5 * m[11] - 0.125 * (m[6] + m[7]);
        const Vec<NV, R> u16 = 0.25 * (u[2] + u[6] + u[10] + u[12] + m[12] + m[14]) + 0.5 * m[11] - 0.125 * (m[5] + m[7]);
        const Vec<NV, R> u18 = 0.25 * (u[4] + u[8] + u[10] + u[11] + m[12] + m[15]) + 0.5 * m[11] - 0.125 * (m[5] + m[6]);
        const Vec<NV, R> ssum = source_at(u14, *src) + source_at(u14 - m[2] - 0.5 * m[13], *src) +
                                source_at(u16, *src) + source_at(u16 - m[3] - 0.5 * m[14], *src) +
                                source_at(u18, *src) + source_at(u18 - m[4] - 0.5 * m[15], *src);
        const Vec<NV, R> s20 = source_at(u[1] + m[11] + m[12], *src);
        const Vec<NV, R> S11 = 2.0 * (ssum - 6.0 * S1) / 3.0 - s20 + s1;
        const Vec<NV, R> S12 = s20 - s1 - S11;
        *sdt = S1 + 0.5 * S11 + S12 / 3.0;
    }
}

template <int NV, class R>
ADER_DEV void predict_modal_src(Vec<NV, R>* m, R gm1, R cx, R cy, R cz, PredCtl& ctl, const Src<R>& src,
                                Vec<NV, R>& sdt) {
    predict_modal<NV, R, true>(m, gm1, cx, cy, cz, ctl, &src, &sdt);
}

// ------------------------------------------------------------------ nodal, App. B
// SRC: with a non-stiff source (s = dt S at nodes 1-7 once and at the tau > 0
// nodes of the current iterate; the source terms of Eqs. B.2-B.3); sdt
// receives dt S-bar of Eq. B.6 from the source at the final iterate.
template <int NV, class R, bool SRC = false>
ADER_DEV void predict_nodal(Vec<NV, R>* m, R gm1, R cx, R cy, R cz, PredCtl& ctl, const Src<R>* src = nullptr,
                            Vec<NV, R>* sdt = nullptr) {
    // Eq. B.4: the ten tau = 0 nodes of Eq. B.1
    Vec<NV, R> u[16];
    u[1] = m[1] - (m[5] + m[6] + m[7]) / 12.0;
    u[2] = u[1] + 0.5 * m[2] + 0.25 * m[5];
    u[3] = 2.0 * u[1] - u[2] + 0.5 * m[5];
    u[4] = u[1] + 0.5 * m[3] + 0.25 * m[6];
    u[5] = 2.0 * u[1] - u[4] + 0.5 * m[6];
    u[6] = u[1] + 0.5 * m[4] + 0.25 * m[7];
    u[7] = 2.0 * u[1] - u[6] + 0.5 * m[7];
    u[8] = u[4] + u[6] - u[1] + 0.25 * m[9];
    u[9] = u[2] + u[6] - u[1] + 0.25 * m[10];
    u[10] = u[2] + u[4] - u[1] + 0.25 * m[8];
    // scaled fluxes at the tau = 0 nodes the q-terms of Eq. B.2 use
    Vec<NV, R> f[11], g[11], h[11];
#pragma unroll
    for (int n = 1; n <= 10; ++n) {
        const Prim<NV, R> q = primitives(u[n], gm1);
        f[n] = scale(cx, flux_from<0>(u[n], q));
        g[n] = scale(cy, flux_from<1>(u[n], q));
        h[n] = scale(cz, flux_from<2>(u[n], q));
    }
    // Eq. B.2 without sources
    Vec<NV, R> q11 = u[1] + 0.5 * (f[3] - f[1]) + 0.5 * (g[5] - g[1]) + 0.5 * (h[7] - h[1]);
    Vec<NV, R> q12 = u[2] + (36.0 * f[1] - 24.0 * f[2] - 12.0 * f[3] - 36.0 * g[1] + 24.0 * g[2] + 24.0 * g[4] +
                             12.0 * g[5] - 24.0 * g[10] - 36.0 * h[1] + 24.0 * h[2] + 24.0 * h[6] + 12.0 * h[7] -
                             24.0 * h[9]) / 24.0;
    Vec<NV, R> q13 = u[4] + (-36.0 * f[1] + 24.0 * f[2] + 12.0 * f[3] + 24.0 * f[4] - 24.0 * f[10] + 36.0 * g[1] -
                             24.0 * g[4] - 12.0 * g[5] - 36.0 * h[1] + 24.0 * h[4] + 24.0 * h[6] + 12.0 * h[7] -
                             24.0 * h[8]) / 24.0;
    Vec<NV, R> q14 = u[6] + (-36.0 * f[1] + 24.0 * f[2] + 12.0 * f[3] + 24.0 * f[6] - 24.0 * f[9] - 36.0 * g[1] +
                             24.0 * g[4] + 12.0 * g[5] + 24.0 * g[6] - 24.0 * g[8] + 36.0 * h[1] - 24.0 * h[6] -
                             12.0 * h[7]) / 24.0;
    Vec<NV, R> q15 = u[1] + (-60.0 * f[1] + 30.0 * f[2] + 30.0 * f[3] - 60.0 * g[1] + 30.0 * g[4] + 30.0 * g[5] -
                             60.0 * h[1] + 30.0 * h[6] + 30.0 * h[7]) / 30.0;
    Vec<NV, R> s0sum, s1;         // with a source: s2 + ... + s7 and s1 (nodes 1-7, built once)
    if constexpr (SRC) {          // Eq. B.2, source terms
        Vec<NV, R> sn[8];
#pragma unroll
        for (int n = 1; n <= 7; ++n) sn[n] = source_at(u[n], *src);
        s1 = sn[1];
        s0sum = sn[2] + sn[3] + sn[4] + sn[5] + sn[6] + sn[7];
        q11 += (-9.0 * sn[1] + 2.0 * s0sum) / 24.0;
        q12 += (7.0 * sn[1] - 10.0 * sn[2] - 6.0 * sn[3] + 2.0 * s0sum) / 24.0;
        q13 += (7.0 * sn[1] - 10.0 * sn[4] - 6.0 * sn[5] + 2.0 * s0sum) / 24.0;
        q14 += (7.0 * sn[1] - 10.0 * sn[6] - 6.0 * sn[7] + 2.0 * s0sum) / 24.0;
        q15 += (-27.0 * sn[1] + 5.0 * s0sum) / 30.0;
    }
    // initial guess: the evolutionary modes in m[11..15] (zero: no time evolution) at the
    // tau > 0 nodes of Eq. B.1
    const Vec<NV, R> g0 = 0.5 * m[11] + 0.25 * m[12];
    Vec<NV, R> u11 = u[1] + g0, u12 = u[2] + g0 + 0.25 * m[13], u13 = u[4] + g0 + 0.25 * m[14];
    Vec<NV, R> u14 = u[6] + g0 + 0.25 * m[15], u15 = u[1] + m[11] + m[12];
    const bool conv = positive_arg(ctl.tol);
    const int cap = conv ? ctl.max_iter : ctl.n_iter;
    const R ref = max_abs(m[1]) + R(sizeof(R) == 8 ? 1e-300 : 1e-30);   // never zero in R
    ctl.iters = 0;
    ctl.capped = conv;
    for (int it = 0; it < cap; ++it) {
        // Eq. B.3 without sources (node 15 serves only source terms)
        const Prim<NV, R> p11 = primitives(u11, gm1);
        const Vec<NV, R> q1 = 0.5 * (scale(cx, flux_from<0>(u11, p11) - flux<0>(u12, gm1)) +
                               scale(cy, flux_from<1>(u11, p11) - flux<1>(u13, gm1)) +
                               scale(cz, flux_from<2>(u11, p11) - flux<2>(u14, gm1)));
        if constexpr (SRC) {      // Eq. B.3 with its source terms, at the current iterate
            const Vec<NV, R> s11 = source_at(u11, *src), s12 = source_at(u12, *src);
            const Vec<NV, R> s13 = source_at(u13, *src), s14 = source_at(u14, *src), s15 = source_at(u15, *src);
            const Vec<NV, R> q2 = q1 + (-4.0 * s11 - 3.0 * s15) / 24.0;
            u11 = q11 + q1 + 0.125 * (4.0 * s11 - s15);
            u12 = q12 + q2 + (2.0 / 3.0) * s12;
            u13 = q13 + q2 + (2.0 / 3.0) * s13;
            u14 = q14 + q2 + (2.0 / 3.0) * s14;
            u15 = q15 + 4.0 * q1 + 0.1 * (8.0 * s11 + s15);
        } else {
            u11 = q11 + q1;
            u12 = q12 + q1;
            u13 = q13 + q1;
            u14 = q14 + q1;
            u15 = q15 + 4.0 * q1;
        }
        ++ctl.iters;
        if (conv) {
            // Eq. B.5 each iteration, to measure the change in mode space
            const Vec<NV, R> n12 = 2.0 * (u15 - 2.0 * u11 + u[1]);
            const Vec<NV, R> n11 = 2.0 * (u11 - u[1] - 0.25 * n12);
            const Vec<NV, R> n13 = 4.0 * (u12 - u11 - u[2] + u[1]);
            const Vec<NV, R> n14 = 4.0 * (u13 - u11 - u[4] + u[1]);
            const Vec<NV, R> n15 = 4.0 * (u14 - u11 - u[6] + u[1]);
            const R change = fmax(fmax(fmax(max_abs_diff(n11, m[11]), max_abs_diff(n12, m[12])),
                                       fmax(max_abs_diff(n13, m[13]), max_abs_diff(n14, m[14]))),
                                  max_abs_diff(n15, m[15]));
            m[11] = n11;
            m[12] = n12;
            m[13] = n13;
            m[14] = n14;
            m[15] = n15;
            if (change < R(ctl.tol) * ref) {
                ctl.capped = false;
                break;
            }
        }
    }
    if (!conv) {
        // Eq. B.5: nodal -> modal
        m[12] = 2.0 * (u15 - 2.0 * u11 + u[1]);
        m[11] = 2.0 * (u11 - u[1] - 0.25 * m[12]);
        m[13] = 4.0 * (u12 - u11 - u[2] + u[1]);
        m[14] = 4.0 * (u13 - u11 - u[4] + u[1]);
        m[15] = 4.0 * (u14 - u11 - u[6] + u[1]);
    }
    if constexpr (SRC)            // Eq. B.6 from the source at the final iterate (times dt)
        *sdt = (-5.0 * s1 + s0sum + 4.0 * source_at(u11, *src) + source_at(u15, *src)) / 6.0;
}

template <int NV, class R>
ADER_DEV void predict_nodal_src(Vec<NV, R>* m, R gm1, R cx, R cy, R cz, PredCtl& ctl, const Src<R>& src,
                                Vec<NV, R>& sdt) {
    predict_nodal<NV, R, true>(m, gm1, cx, cy, cz, ctl, &src, &sdt);
}

constexpr bool HAS_SOURCE = true;
constexpr bool HAS_SOURCE_MODAL = true;

// ------------------------------------------------------------------ x+ face, Sec. V.2 and App. D
// p = the zone's modes in the face's x-frame (modes.cuh).  Outputs the
// barycentre state (Eq. 61), the face average of u (Eq. 62) and the face
// average of the physical normal flux: composing Eq. D.9 with D.10 gives
// <F> = (F1 + F6 + F7 + F8 + F9 + F10) / 6 over the facial nodes of Eq. D.6
// (the four corner nodes enter only the edge averages).
template <int D, int NV, class R>
ADER_DEV void face(const Vec<NV, R>* p, R gm1, Vec<NV, R>& ub, Vec<NV, R>& avg, Vec<NV, R>& Fa) {
    ub = p[1] + 0.5 * (p[2] + p[11]) + 0.25 * (p[12] + p[13]) + (2.0 * p[5] - p[6] - p[7]) / 12.0;
    avg = ub + (p[6] + p[7] + p[12]) / 12.0;
    // Eq. D.8
    const Vec<NV, R> q1 = 0.5 * p[11] + 0.25 * (p[12] + p[13]);
    const Vec<NV, R> t1 = p[1] + 0.5 * p[2] + (2.0 * p[5] - p[6] - p[7]) / 12.0;
    const Vec<NV, R> t2 = t1 + 0.5 * (p[3] + p[4]) + 0.25 * (p[6] + p[7] + p[8] + p[9] + p[10]);
    const Vec<NV, R> t3 = t2 - p[3] - 0.5 * (p[8] + p[9]);
    const Vec<NV, R> t4 = t2 - p[4] - 0.5 * (p[9] + p[10]);
    const Vec<NV, R> t5 = t4 - p[3] - 0.5 * (p[8] - p[9]);
    const Vec<NV, R> t6 = 0.5 * (t2 + t4) + q1 + 0.25 * (p[14] - p[7]);
    const Vec<NV, R> t7 = 0.5 * (t3 + t5) + q1 - 0.25 * (p[7] + p[14]);
    const Vec<NV, R> t8 = 0.5 * (t2 + t3) + q1 + 0.25 * (p[15] - p[6]);
    const Vec<NV, R> t9 = 0.5 * (t4 + t5) + q1 - 0.25 * (p[6] + p[15]);
    const Vec<NV, R> t10 = t1 + p[11] + p[12] + 0.5 * p[13];
    Fa = (flux<D>(t1, gm1) + flux<D>(t6, gm1) + flux<D>(t7, gm1) + flux<D>(t8, gm1) + flux<D>(t9, gm1) +
          flux<D>(t10, gm1)) / 6.0;
}

// Both x-faces of one direction at once (Euler).  p is the zone's modes in
// the frame of the upper face; the lower face's frame differs only in the
// sign of the modes odd in the normal coordinate (2, 8, 10, 13), so each of
// face()'s node states is E + O on the upper face and E - O on the lower one,
// with E its part from the even modes and O from the odd ones.  E and O are
// face()'s own linear combinations split by parity, each computed once; the
// nodes are taken in an order that keeps few of them alive at a time.
// Index 0 of ub, avg, Fa is the upper face (S = +1), index 1 the lower.
constexpr bool HAS_FACE_PAIR = true;

template <int D, int NV, class R>
ADER_DEV void face_pair(const Vec<NV, R>* p, R gm1, Vec<NV, R>* ub, Vec<NV, R>* avg, Vec<NV, R>* Fa) {
    const Vec<NV, R> t1e = p[1] + (2.0 * p[5] - p[6] - p[7]) / 12.0, t1o = 0.5 * p[2];
    const Vec<NV, R> q1e = 0.5 * p[11] + 0.25 * p[12], q1o = 0.25 * p[13];
    {
        const Vec<NV, R> ube = t1e + q1e, ubo = t1o + q1o;
        const Vec<NV, R> avge = ube + (p[6] + p[7] + p[12]) / 12.0;
        ub[0] = ube + ubo;
        ub[1] = ube - ubo;
        avg[0] = avge + ubo;
        avg[1] = avge - ubo;
    }
    Vec<NV, R> up = flux<D>(t1e + t1o, gm1), lo = flux<D>(t1e - t1o, gm1);       // node 1
    {
        const Vec<NV, R> e = t1e + p[11] + p[12], o = t1o + 0.5 * p[13];          // node 10
        up += flux<D>(e + o, gm1);
        lo += flux<D>(e - o, gm1);
    }
    const Vec<NV, R> t2e = t1e + 0.5 * (p[3] + p[4]) + 0.25 * (p[6] + p[7] + p[9]), t2o = t1o + 0.25 * (p[8] + p[10]);
    const Vec<NV, R> t3e = t2e - p[3] - 0.5 * p[9], t3o = t2o - 0.5 * p[8];
    const Vec<NV, R> t4e = t2e - p[4] - 0.5 * p[9], t4o = t2o - 0.5 * p[10];
    {
        const Vec<NV, R> e = 0.5 * (t2e + t4e) + q1e + 0.25 * (p[14] - p[7]), o = 0.5 * (t2o + t4o) + q1o;   // 6
        up += flux<D>(e + o, gm1);
        lo += flux<D>(e - o, gm1);
    }
    {
        const Vec<NV, R> e = 0.5 * (t2e + t3e) + q1e + 0.25 * (p[15] - p[6]), o = 0.5 * (t2o + t3o) + q1o;   // 8
        up += flux<D>(e + o, gm1);
        lo += flux<D>(e - o, gm1);
    }
    const Vec<NV, R> t5e = t4e - p[3] + 0.5 * p[9], t5o = t4o - 0.5 * p[8];
    {
        const Vec<NV, R> e = 0.5 * (t4e + t5e) + q1e - 0.25 * (p[6] + p[15]), o = 0.5 * (t4o + t5o) + q1o;   // 9
        up += flux<D>(e + o, gm1);
        lo += flux<D>(e - o, gm1);
    }
    {
        const Vec<NV, R> e = 0.5 * (t3e + t5e) + q1e - 0.25 * (p[7] + p[14]), o = 0.5 * (t3o + t5o) + q1o;   // 7
        up += flux<D>(e + o, gm1);
        lo += flux<D>(e - o, gm1);
    }
    Fa[0] = up / 6.0;
    Fa[1] = lo / 6.0;
}

// MHD face: all ten facial nodes of Eq. D.6; edge averages by Eq. 63 (<u>)
// and Eqs. D.9-D.10 (<F>) for the field component of each edge's EMF
// (slots t1+, t1-, t2+, t2-; component 5 + t1 / 5 + t2).
template <int D, class R>
ADER_DEV void face_mhd(const Vec<8, R>* p, R gm1, Vec<8, R>& ub, Vec<8, R>& avg, Vec<8, R>& Fa, R* eu, R* ef) {
    constexpr int T1 = D == 0 ? 1 : 0, T2 = D == 2 ? 1 : 2;
    ub = p[1] + 0.5 * (p[2] + p[11]) + 0.25 * (p[12] + p[13]) + (2.0 * p[5] - p[6] - p[7]) / 12.0;
    avg = ub + (p[6] + p[7] + p[12]) / 12.0;
    Vec<8, R> t[11];
    const Vec<8, R> q1 = 0.5 * p[11] + 0.25 * (p[12] + p[13]);
    t[1] = p[1] + 0.5 * p[2] + (2.0 * p[5] - p[6] - p[7]) / 12.0;
    t[2] = t[1] + 0.5 * (p[3] + p[4]) + 0.25 * (p[6] + p[7] + p[8] + p[9] + p[10]);
    t[3] = t[2] - p[3] - 0.5 * (p[8] + p[9]);
    t[4] = t[2] - p[4] - 0.5 * (p[9] + p[10]);
    t[5] = t[4] - p[3] - 0.5 * (p[8] - p[9]);
    t[6] = 0.5 * (t[2] + t[4]) + q1 + 0.25 * (p[14] - p[7]);
    t[7] = 0.5 * (t[3] + t[5]) + q1 - 0.25 * (p[7] + p[14]);
    t[8] = 0.5 * (t[2] + t[3]) + q1 + 0.25 * (p[15] - p[6]);
    t[9] = 0.5 * (t[4] + t[5]) + q1 - 0.25 * (p[6] + p[15]);
    t[10] = t[1] + p[11] + p[12] + 0.5 * p[13];
    Vec<8, R> F[11];
#pragma unroll
    for (int n = 1; n <= 10; ++n) F[n] = flux<D>(t[n], gm1);
    Fa = (F[1] + F[6] + F[7] + F[8] + F[9] + F[10]) / 6.0;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const int c = 5 + (s == 0 ? T1 : T2);
        auto f = [&](int n) { return F[n][c]; };
        // Eq. D.9 (the modes the edge averages need)
        const R q2 = R(0.5) * (f(2) + f(4) - R(4) * f(1) + f(3) + f(5));
        const R q3 = f(6) + f(7) - f(8) - f(9);
        const R m1 = R(2.0 / 3.0) * (f(1) + R(0.125) * (f(2) + f(3) + f(4) + f(5)));
        const R m2 = R(0.5) * (f(2) + f(4) - f(3) - f(5));
        const R m3 = R(0.5) * (f(2) + f(3) - f(4) - f(5));
        const R m4 = q2 + q3, m5 = q2 - q3;
        const R m8 = R(2) * (f(1) + f(10)) - (f(6) + f(7) + f(8) + f(9)) + q2;
        const R m7 = f(10) - f(1) - m8;
        const R m9 = R(2) * (f(6) - f(7) - m2);
        const R m10 = R(2) * (f(8) - f(9) - m3);
        // Eq. D.10
        const R af = m1 + R(0.5) * m7 + m8 * R(1.0 / 3.0);
        const R qs = s == 0 ? R(0.5) * m2 + R(0.25) * m9 : R(0.5) * m3 + R(0.25) * m10;
        const R plus = af + qs + (s == 0 ? m4 : m5) * R(1.0 / 6.0);
        ef[2 * s] = plus;
        ef[2 * s + 1] = plus - R(2) * qs;
        // Eq. 63
        const R qu = s == 0 ? R(0.5) * p[3][c] + R(0.25) * (p[8][c] + p[14][c])
                            : R(0.5) * p[4][c] + R(0.25) * (p[10][c] + p[15][c]);
        const R up = avg[c] + (s == 0 ? p[6][c] : p[7][c]) * R(1.0 / 6.0) + qu;
        eu[2 * s] = up;
        eu[2 * s + 1] = up - R(2) * qu;
    }
}

// Full edge-averaged states (all eight components; Eq. 63) for the
// linearized edge fluxes.  Slots as in face_mhd.
template <int D, class R>
ADER_DEV void edge_states(const Vec<8, R>* p, const Vec<8, R>& ub, const Vec<8, R>& avg, Vec<8, R>* e) {
    (void)ub;
    const Vec<8, R> q1 = 0.5 * p[3] + 0.25 * (p[8] + p[14]), q2 = 0.5 * p[4] + 0.25 * (p[10] + p[15]);
    const Vec<8, R> u1 = avg + p[6] / 6.0 + q1, u2 = avg + p[7] / 6.0 + q2;
    e[0] = u1;
    e[1] = u1 - 2.0 * q1;
    e[2] = u2;
    e[3] = u2 - 2.0 * q2;
}

}  // namespace o3
}  // namespace ader
