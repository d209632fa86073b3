// Fourth order: ADER-CG predictor (modal Sec. IV.3, nodal App. C) and the x+
// face quantities (Sec. V.3, App. D).  Modes m[1..35] (Eq. 16).
#pragma once
#include "common.cuh"
#include "modes.cuh"
#include "nodal_o4_coeffs.cuh"

namespace ader {
namespace o4 {


// ------------------------------------------------------------------ modal, Sec. IV.3
// SRC: with a non-stiff source (s = dt S at every node of Eq. 46 of the current iterate; the source
// modes by Eqs. 49-51 with f, g, h -> s and Eq. 52; Eq. 45 with its source terms); sdt receives dt S-bar
// of Eq. 53 from the final iterate.
template <int NV, class R, bool SRC = false>
ADER_DEV void predict_modal(Vec<NV, R>* m, R gm1, R cx, R cy, R cz, PredCtl& ctl, const Src<R>* src = nullptr,
                            Vec<NV, R>* sdt = nullptr) {
    // Eq. 47: the 21 tau = 0 nodes of Eq. 46
    Vec<NV, R> u[22];
    u[1] = m[1] - (m[5] + m[6] + m[7]) / 12.0;
    u[2] = u[1] + (60.0 * m[2] + 30.0 * m[5] + 6.0 * m[11] - 5.0 * m[16] - 5.0 * m[18]) / 120.0;
    u[3] = 0.5 * (u[1] + u[2]) - 0.015625 * (4.0 * m[5] + 3.0 * m[11]);
    u[4] = 3.0 * u[1] + u[2] - 3.0 * u[3] - 0.09375 * m[11];
    u[5] = 6.0 * u[1] + 3.0 * u[2] - 8.0 * u[3] - 0.375 * m[11];
    u[6] = u[1] + (60.0 * m[3] + 30.0 * m[6] + 6.0 * m[12] - 5.0 * m[14] - 5.0 * m[19]) / 120.0;
    u[7] = 0.5 * (u[1] + u[6]) - 0.015625 * (4.0 * m[6] + 3.0 * m[12]);
    u[8] = 3.0 * u[1] + u[6] - 3.0 * u[7] - 0.09375 * m[12];
    u[9] = 6.0 * u[1] + 3.0 * u[6] - 8.0 * u[7] - 0.375 * m[12];
    u[10] = u[1] + (60.0 * m[4] + 30.0 * m[7] + 6.0 * m[13] - 5.0 * m[15] - 5.0 * m[17]) / 120.0;
    u[11] = 0.5 * (u[1] + u[10]) - 0.015625 * (4.0 * m[7] + 3.0 * m[13]);
    u[12] = 3.0 * u[1] + u[10] - 3.0 * u[11] - 0.09375 * m[13];
    u[13] = 6.0 * u[1] + 3.0 * u[10] - 8.0 * u[11] - 0.375 * m[13];
    u[14] = u[2] + u[7] + u[10] - 2.0 * u[1] + 0.25 * (m[3] + m[8] + m[9] + m[10]) + (5.0 / 48.0) * (m[14] + m[19]) +
            (23.0 / 320.0) * m[12] + 0.125 * (m[15] + m[16] + m[17] + m[18] + m[20]) + 0.1875 * m[6];
    u[15] = u[14] + u[9] - u[6] - 0.5 * (m[8] + m[9]) - 0.25 * (m[14] + m[19] + m[20]);
    u[16] = u[14] + u[13] - u[10] - 0.5 * (m[9] + m[10]) - 0.25 * (m[15] + m[17] + m[20]);
    u[18] = u[14] + u[5] - u[2] - 0.5 * (m[8] + m[10]) - 0.25 * (m[16] + m[18] + m[20]);
    u[19] = u[18] + u[9] - u[6] + 0.5 * (m[8] - m[9]) - 0.25 * (m[14] + m[19] - m[20]);
    u[20] = u[18] + u[13] - u[10] - 0.5 * (m[9] - m[10]) - 0.25 * (m[15] + m[17] - m[20]);
    u[17] = u[15] + u[16] - u[14] + m[9] + 0.5 * m[20];
    u[21] = u[19] + u[20] - u[18] + m[9] - 0.5 * m[20];

    // tau = 0 parts of Eqs. 49-51 (built once)
    Vec<NV, R> F2, F5, F8, F10, F11, F20, PF14, PF15, PF16, QF12;
    Vec<NV, R> G3, G6, G8, G9, G12, G20, PG14, PG15, PG16, QG34;
    Vec<NV, R> H4, H7, H9, H10, H13, H20, PH14, PH15, PH16, QH56;
    {
        Vec<NV, R> f[22], g[22], h[22];
#pragma unroll
        for (int n = 1; n <= 21; ++n) {
            const Prim<NV, R> q = primitives(u[n], gm1);
            f[n] = flux_from<0>(u[n], q);
            g[n] = flux_from<1>(u[n], q);
            h[n] = flux_from<2>(u[n], q);
        }
        // q1..q6 of Eqs. 49-51 (corner sums), per flux
        const Vec<NV, R> fq1 = f[14] + f[15] + f[16] + f[17], fq2 = f[18] + f[19] + f[20] + f[21];
        const Vec<NV, R> fq3 = f[14] + f[16] + f[18] + f[20], fq4 = f[15] + f[17] + f[19] + f[21];
        const Vec<NV, R> fq5 = f[14] + f[15] + f[18] + f[19], fq6 = f[16] + f[17] + f[20] + f[21];
        F5 = 2.0 * (f[2] - 2.0 * f[1] + f[5]);
        F8 = 0.5 * (f[14] - f[15] + f[16] - f[17] - f[18] + f[19] - f[20] + f[21]);
        F10 = 0.5 * (f[14] + f[15] - f[16] - f[17] - f[18] - f[19] + f[20] + f[21]);
        F11 = (16.0 / 3.0) * (f[2] - 2.0 * f[3] + 2.0 * f[4] - f[5]);
        F2 = (2.0 / 3.0) * (f[2] - f[5]) - 0.1 * F11 + (fq1 - fq2) / 12.0;
        F20 = f[14] - f[15] - f[16] + f[17] - f[18] + f[19] + f[20] - f[21];
        PF14 = 0.5 * (fq3 - fq4) - 2.0 * (f[6] - f[9]);
        PF15 = 0.5 * (fq5 - fq6) - 2.0 * (f[10] - f[13]);
        PF16 = 0.5 * (fq1 - fq2) - 2.0 * (f[2] - f[5]);
        QF12 = fq1 - fq2;
        const Vec<NV, R> gq1 = g[14] + g[15] + g[16] + g[17], gq2 = g[18] + g[19] + g[20] + g[21];
        const Vec<NV, R> gq3 = g[14] + g[16] + g[18] + g[20], gq4 = g[15] + g[17] + g[19] + g[21];
        const Vec<NV, R> gq5 = g[14] + g[15] + g[18] + g[19], gq6 = g[16] + g[17] + g[20] + g[21];
        G6 = 2.0 * (g[6] - 2.0 * g[1] + g[9]);
        G8 = 0.5 * (g[14] - g[15] + g[16] - g[17] - g[18] + g[19] - g[20] + g[21]);
        G9 = 0.5 * (g[14] - g[15] - g[16] + g[17] + g[18] - g[19] - g[20] + g[21]);
        G12 = (16.0 / 3.0) * (g[6] - 2.0 * g[7] + 2.0 * g[8] - g[9]);
        G3 = (2.0 / 3.0) * (g[6] - g[9]) - 0.1 * G12 + (gq3 - gq4) / 12.0;
        G20 = g[14] - g[15] - g[16] + g[17] - g[18] + g[19] + g[20] - g[21];
        PG14 = 0.5 * (gq3 - gq4) - 2.0 * (g[6] - g[9]);
        PG15 = 0.5 * (gq5 - gq6) - 2.0 * (g[10] - g[13]);
        PG16 = 0.5 * (gq1 - gq2) - 2.0 * (g[2] - g[5]);
        QG34 = gq3 - gq4;
        const Vec<NV, R> hq1 = h[14] + h[15] + h[16] + h[17], hq2 = h[18] + h[19] + h[20] + h[21];
        const Vec<NV, R> hq3 = h[14] + h[16] + h[18] + h[20], hq4 = h[15] + h[17] + h[19] + h[21];
        const Vec<NV, R> hq5 = h[14] + h[15] + h[18] + h[19], hq6 = h[16] + h[17] + h[20] + h[21];
        H7 = 2.0 * (h[10] - 2.0 * h[1] + h[13]);
        H9 = 0.5 * (h[14] - h[15] - h[16] + h[17] + h[18] - h[19] - h[20] + h[21]);
        H10 = 0.5 * (h[14] + h[15] - h[16] - h[17] - h[18] - h[19] + h[20] + h[21]);
        H13 = (16.0 / 3.0) * (h[10] - 2.0 * h[11] + 2.0 * h[12] - h[13]);
        H4 = (2.0 / 3.0) * (h[10] - h[13]) - 0.1 * H13 + (hq5 - hq6) / 12.0;
        H20 = h[14] - h[15] - h[16] + h[17] - h[18] + h[19] + h[20] - h[21];
        PH14 = 0.5 * (hq3 - hq4) - 2.0 * (h[6] - h[9]);
        PH15 = 0.5 * (hq5 - hq6) - 2.0 * (h[10] - h[13]);
        PH16 = 0.5 * (hq1 - hq2) - 2.0 * (h[2] - h[5]);
        QH56 = hq5 - hq6;
    }
    // source modes from the tau = 0 nodes (Eqs. 49-52 with f, g, h -> s), built once
    Vec<NV, R> s1, S1, S2, S3, S4, S5, S6, S7, S8, S9, S10, PS14, PS15, PS16, QS12, QS34, QS56;
    if constexpr (SRC) {
        Vec<NV, R> sn[22];
#pragma unroll
        for (int k = 1; k <= 21; ++k) sn[k] = source_at(u[k], *src);
        const Vec<NV, R> a1 = sn[14] + sn[15] + sn[16] + sn[17], a2 = sn[18] + sn[19] + sn[20] + sn[21];
        const Vec<NV, R> a3 = sn[14] + sn[16] + sn[18] + sn[20], a4 = sn[15] + sn[17] + sn[19] + sn[21];
        const Vec<NV, R> a5 = sn[14] + sn[15] + sn[18] + sn[19], a6 = sn[16] + sn[17] + sn[20] + sn[21];
        s1 = sn[1];
        S5 = 2.0 * (sn[2] - 2.0 * sn[1] + sn[5]);
        S6 = 2.0 * (sn[6] - 2.0 * sn[1] + sn[9]);
        S7 = 2.0 * (sn[10] - 2.0 * sn[1] + sn[13]);
        S8 = 0.5 * (sn[14] - sn[15] + sn[16] - sn[17] - sn[18] + sn[19] - sn[20] + sn[21]);
        S9 = 0.5 * (sn[14] - sn[15] - sn[16] + sn[17] + sn[18] - sn[19] - sn[20] + sn[21]);
        S10 = 0.5 * (sn[14] + sn[15] - sn[16] - sn[17] - sn[18] - sn[19] + sn[20] + sn[21]);
        const Vec<NV, R> S11 = (16.0 / 3.0) * (sn[2] - 2.0 * sn[3] + 2.0 * sn[4] - sn[5]);
        const Vec<NV, R> S12 = (16.0 / 3.0) * (sn[6] - 2.0 * sn[7] + 2.0 * sn[8] - sn[9]);
        const Vec<NV, R> S13 = (16.0 / 3.0) * (sn[10] - 2.0 * sn[11] + 2.0 * sn[12] - sn[13]);
        S2 = (2.0 / 3.0) * (sn[2] - sn[5]) - 0.1 * S11 + (a1 - a2) / 12.0;
        S3 = (2.0 / 3.0) * (sn[6] - sn[9]) - 0.1 * S12 + (a3 - a4) / 12.0;
        S4 = (2.0 / 3.0) * (sn[10] - sn[13]) - 0.1 * S13 + (a5 - a6) / 12.0;
        PS14 = 0.5 * (a3 - a4) - 2.0 * (sn[6] - sn[9]);
        PS15 = 0.5 * (a5 - a6) - 2.0 * (sn[10] - sn[13]);
        PS16 = 0.5 * (a1 - a2) - 2.0 * (sn[2] - sn[5]);
        QS12 = a1 - a2;
        QS34 = a3 - a4;
        QS56 = a5 - a6;
        S1 = 0.125 * (a1 + a2) - (S5 + S6 + S7) / 6.0;
    }
    // the time modes of the source (Eqs. 49-52 with f, g, h -> s) from the nodes 22..42 of an iterate
    auto time_source_modes = [&](const Vec<NV, R>* w, Vec<NV, R>* T) {
        Vec<NV, R> sw[43];
#pragma unroll
        for (int k = 22; k <= 42; ++k) sw[k] = source_at(w[k], *src);
        const Vec<NV, R> q7 = sw[23] + sw[24] - sw[25] - sw[26] - sw[27] - sw[28] + sw[29] + sw[30];
        const Vec<NV, R> q8 = sw[23] + sw[27] - sw[24] - sw[28] - sw[31] - sw[33] + sw[32] + sw[34];
        const Vec<NV, R> q9 = sw[25] + sw[29] - sw[26] - sw[30] - sw[31] - sw[32] + sw[33] + sw[34];
        const Vec<NV, R> q10 = sw[23] + sw[24] + sw[25] + sw[26] - sw[27] - sw[28] - sw[29] - sw[30];
        const Vec<NV, R> q11 = sw[23] - sw[24] + sw[27] - sw[28] + sw[31] - sw[32] + sw[33] - sw[34];
        const Vec<NV, R> q12 = sw[25] - sw[26] + sw[29] - sw[30] + sw[31] + sw[32] - sw[33] - sw[34];
        const Vec<NV, R> S16 = q7 + PS16, S18 = -2.0 * q7 + S16;
        const Vec<NV, R> S14 = q8 + PS14, S19 = -2.0 * q8 + S14;
        const Vec<NV, R> S15 = q9 + PS15, S17 = -2.0 * q9 + S15;
        // T[k - 21] = s mode k for k = 21..35
        T[6] = 1.125 * QS12 + 4.5 * (sw[36] - sw[37]) - 2.25 * q10;                               // 27
        T[3] = 3.0 * (sw[36] - sw[37]) - 0.75 * q10 + 0.375 * (S16 + S18) - T[6];                // 24
        T[7] = 1.125 * QS34 + 4.5 * (sw[38] - sw[39]) - 2.25 * q11;                               // 28
        T[4] = 3.0 * (sw[38] - sw[39]) - 0.75 * q11 + 0.375 * (S14 + S19) - T[7];                // 25
        T[8] = 1.125 * QS56 + 4.5 * (sw[40] - sw[41]) - 2.25 * q12;                               // 29
        T[5] = 3.0 * (sw[40] - sw[41]) - 0.75 * q12 + 0.375 * (S15 + S17) - T[8];                // 26
        T[9] = 3.0 * (sw[36] - 2.0 * sw[35] + sw[37]) - 1.5 * S5;                                // 30
        T[10] = 3.0 * (sw[38] - 2.0 * sw[35] + sw[39]) - 1.5 * S6;                               // 31
        T[11] = 3.0 * (sw[40] - 2.0 * sw[35] + sw[41]) - 1.5 * S7;                               // 32
        T[12] = 3.0 * (sw[23] - sw[27] - sw[24] + sw[28]) - 3.0 * S8;                            // 33
        T[13] = 3.0 * (sw[31] - sw[32] - sw[33] + sw[34]) - 3.0 * S9;                            // 34
        T[14] = 3.0 * (sw[25] - sw[29] - sw[26] + sw[30]) - 3.0 * S10;                           // 35
        T[2] = 4.5 * (sw[42] - s1) - 13.5 * (sw[35] - sw[22]);                                   // 23 (Eq. 52)
        T[1] = 2.25 * (s1 - sw[22] - sw[35] + sw[42]) - 1.5 * T[2];                              // 22
        T[0] = sw[42] - s1 - T[1] - T[2] + (T[9] + T[10] + T[11]) / 12.0;                        // 21
    };
    // Eq. 48: the tau > 0 nodes 22..41 of Eq. 46 of the current iterate (22 and 42 serve only source
    // terms; 42 = (0, 0, 0, 1) only with a source)
    auto build_w = [&](Vec<NV, R>* w) {
        w[22] = u[1] + (36.0 * m[21] + 12.0 * m[22] + 4.0 * m[23] - 3.0 * m[30] - 3.0 * m[31] - 3.0 * m[32]) / 108.0;
        w[23] = w[22] + u[2] + u[6] - 2.0 * u[1] +
                (18.0 * m[8] + 9.0 * m[14] + 9.0 * m[16] + 12.0 * m[24] + 12.0 * m[25] + 4.0 * m[27] + 4.0 * m[28] +
                 6.0 * m[30] + 6.0 * m[31] + 6.0 * m[33]) / 72.0;
        w[24] = w[23] - u[6] + u[9] - 0.5 * m[8] - 0.25 * m[14] - (6.0 * m[25] + 2.0 * m[28] + 3.0 * m[33]) / 18.0;
        w[25] = 0.5 * (u[14] + u[15] + w[23] + w[24]) - u[2] - 0.5 * m[6] - 0.25 * m[16] - 0.125 * m[17] +
                (6.0 * m[26] + 2.0 * m[29] - 3.0 * m[31] + 3.0 * m[32] + 3.0 * m[35]) / 36.0;
        w[26] = w[23] + w[24] - w[25] - 0.5 * (m[6] - m[7]) - 0.25 * (m[16] - m[18]) - (m[31] - m[32]) / 6.0;
        w[27] = u[5] + w[23] - u[2] - 0.5 * m[8] - 0.25 * m[16] - (6.0 * m[24] + 2.0 * m[27] + 3.0 * m[33]) / 18.0;
        w[28] = u[9] + w[27] - u[6] + 0.5 * m[8] - 0.25 * m[14] - (6.0 * m[25] + 2.0 * m[28] - 3.0 * m[33]) / 18.0;
        w[29] = 0.5 * (u[18] + u[19] + w[27] + w[28]) - u[5] - 0.5 * m[6] + 0.25 * m[16] - 0.125 * m[17] +
                (6.0 * m[26] + 2.0 * m[29] - 3.0 * m[31] + 3.0 * m[32] - 3.0 * m[35]) / 36.0;
        w[30] = w[27] + w[28] - w[29] - 0.5 * (m[6] - m[7]) + 0.25 * (m[16] - m[18]) - (m[31] - m[32]) / 6.0;
        w[31] = 0.5 * (u[14] + u[18] + w[25] + w[29]) - u[10] - 0.5 * m[5] - 0.25 * m[15] - 0.125 * m[14] +
                (6.0 * m[25] + 2.0 * m[28] - 3.0 * m[30] + 3.0 * m[31] + 3.0 * m[34]) / 36.0;
        w[32] = u[9] + w[31] - u[6] - 0.5 * m[9] - 0.25 * m[19] - (6.0 * m[25] + 2.0 * m[28] + 3.0 * m[34]) / 18.0;
        w[33] = w[23] + w[27] - w[31] - 0.5 * (m[5] - m[7]) - 0.25 * (m[14] - m[19]) - (m[30] - m[32]) / 6.0;
        w[34] = w[24] + w[28] - w[32] - 0.5 * (m[5] - m[7]) + 0.25 * (m[14] - m[19]) - (m[30] - m[32]) / 6.0;
        const Vec<NV, R> r1 = (36.0 * m[21] + 24.0 * m[22] + 16.0 * m[23]) / 54.0;
        const Vec<NV, R> r2 = (18.0 * m[24] + 12.0 * m[27]) / 54.0;
        const Vec<NV, R> r3 = (6.0 * m[30] - 3.0 * m[31] - 3.0 * m[32]) / 54.0;
        const Vec<NV, R> r4 = (18.0 * m[25] + 12.0 * m[28]) / 54.0;
        const Vec<NV, R> r5 = (-3.0 * m[30] + 6.0 * m[31] - 3.0 * m[32]) / 54.0;
        const Vec<NV, R> r6 = (18.0 * m[26] + 12.0 * m[29]) / 54.0;
        const Vec<NV, R> r7 = (-3.0 * m[30] - 3.0 * m[31] + 6.0 * m[32]) / 54.0;
        w[35] = 2.0 * w[22] - u[1] + 2.0 * (m[22] + m[23]) / 9.0;
        w[36] = u[2] + r1 + r2 + r3;
        w[37] = u[5] + r1 - r2 + r3;
        w[38] = u[6] + r1 + r4 + r5;
        w[39] = u[9] + r1 - r4 + r5;
        w[40] = u[10] + r1 + r6 + r7;
        w[41] = u[13] + r1 - r6 + r7;
        if constexpr (SRC) w[42] = u[1] + m[21] + m[22] + m[23] - (m[30] + m[31] + m[32]) / 12.0;   // (0, 0, 0, 1)
    };
    // Eq. 45 without sources: the modes fed by tau = 0 fluxes only
    const Vec<NV, R> e21 = -(scale(cx, F2 + 0.1 * F11) + scale(cy, G3 + 0.1 * G12) + scale(cz, H4 + 0.1 * H13));
    const Vec<NV, R> e24 = -(scale(cx, 2.0 * F5) + scale(cy, G8) + scale(cz, H10));
    const Vec<NV, R> e25 = -(scale(cx, F8) + scale(cy, 2.0 * G6) + scale(cz, H9));
    const Vec<NV, R> e26 = -(scale(cx, F10) + scale(cy, G9) + scale(cz, 2.0 * H7));

    const bool conv = positive_arg(ctl.tol);
    const int cap = conv ? ctl.max_iter : ctl.n_iter;
    const R ref = max_abs(m[1]) + R(sizeof(R) == 8 ? 1e-300 : 1e-30);   // never zero in R
    ctl.iters = 0;
    ctl.capped = conv;
    for (int it = 0; it < cap; ++it) {
        Vec<NV, R> w[43];
        build_w(w);
        // fluxes at nodes 23..35 (all three directions) and the axis nodes 36..41
        Vec<NV, R> f[36], g[36], h[36];
#pragma unroll
        for (int n = 23; n <= 35; ++n) {
            const Prim<NV, R> q = primitives(w[n], gm1);
            f[n] = flux_from<0>(w[n], q);
            g[n] = flux_from<1>(w[n], q);
            h[n] = flux_from<2>(w[n], q);
        }
        const Vec<NV, R> f36 = flux<0>(w[36], gm1), f37 = flux<0>(w[37], gm1);
        const Vec<NV, R> g38 = flux<1>(w[38], gm1), g39 = flux<1>(w[39], gm1);
        const Vec<NV, R> h40 = flux<2>(w[40], gm1), h41 = flux<2>(w[41], gm1);
        // Eq. 49 (x)
        Vec<NV, R> F14, F15, F16, F18, F24, F27, F30, F33, F35;
        {
            const Vec<NV, R> q7 = f[23] + f[24] - f[25] - f[26] - f[27] - f[28] + f[29] + f[30];
            const Vec<NV, R> q8 = f[23] + f[27] - f[24] - f[28] - f[31] - f[33] + f[32] + f[34];
            const Vec<NV, R> q9 = f[25] + f[29] - f[26] - f[30] - f[31] - f[32] + f[33] + f[34];
            const Vec<NV, R> q10 = f[23] + f[24] + f[25] + f[26] - f[27] - f[28] - f[29] - f[30];
            F14 = q8 + PF14;
            F15 = q9 + PF15;
            F16 = q7 + PF16;
            F18 = -2.0 * q7 + F16;
            F27 = 1.125 * QF12 + 4.5 * (f36 - f37) - 2.25 * q10;
            F24 = 3.0 * (f36 - f37) - 0.75 * q10 + 0.375 * (F16 + F18) - F27;
            F30 = 3.0 * (f36 - 2.0 * f[35] + f37) - 1.5 * F5;
            F33 = 3.0 * (f[23] - f[27] - f[24] + f[28]) - 3.0 * F8;
            F35 = 3.0 * (f[25] - f[29] - f[26] + f[30]) - 3.0 * F10;
        }
        // Eq. 50 (y)
        Vec<NV, R> G14, G16, G17, G19, G25, G28, G31, G33, G34;
        {
            const Vec<NV, R> q7 = g[23] + g[24] - g[25] - g[26] - g[27] - g[28] + g[29] + g[30];
            const Vec<NV, R> q8 = g[23] + g[27] - g[24] - g[28] - g[31] - g[33] + g[32] + g[34];
            const Vec<NV, R> q9 = g[25] + g[29] - g[26] - g[30] - g[31] - g[32] + g[33] + g[34];
            const Vec<NV, R> q11 = g[23] - g[24] + g[27] - g[28] + g[31] - g[32] + g[33] - g[34];
            G14 = q8 + PG14;
            const Vec<NV, R> G15 = q9 + PG15;
            G16 = q7 + PG16;
            G17 = -2.0 * q9 + G15;
            G19 = -2.0 * q8 + G14;
            G28 = 1.125 * QG34 + 4.5 * (g38 - g39) - 2.25 * q11;
            G25 = 3.0 * (g38 - g39) - 0.75 * q11 + 0.375 * (G14 + G19) - G28;
            G31 = 3.0 * (g38 - 2.0 * g[35] + g39) - 1.5 * G6;
            G33 = 3.0 * (g[23] - g[27] - g[24] + g[28]) - 3.0 * G8;
            G34 = 3.0 * (g[31] - g[32] - g[33] + g[34]) - 3.0 * G9;
        }
        // Eq. 51 (z)
        Vec<NV, R> H15, H17, H18, H19, H26, H29, H32, H34, H35;
        {
            const Vec<NV, R> q7 = h[23] + h[24] - h[25] - h[26] - h[27] - h[28] + h[29] + h[30];
            const Vec<NV, R> q8 = h[23] + h[27] - h[24] - h[28] - h[31] - h[33] + h[32] + h[34];
            const Vec<NV, R> q9 = h[25] + h[29] - h[26] - h[30] - h[31] - h[32] + h[33] + h[34];
            const Vec<NV, R> q12 = h[25] - h[26] + h[29] - h[30] + h[31] + h[32] - h[33] - h[34];
            const Vec<NV, R> H14 = q8 + PH14;
            H15 = q9 + PH15;
            const Vec<NV, R> H16 = q7 + PH16;
            H17 = -2.0 * q9 + H15;
            H18 = -2.0 * q7 + H16;
            H19 = -2.0 * q8 + H14;
            H29 = 1.125 * QH56 + 4.5 * (h40 - h41) - 2.25 * q12;
            H26 = 3.0 * (h40 - h41) - 0.75 * q12 + 0.375 * (H15 + H17) - H29;
            H32 = 3.0 * (h40 - 2.0 * h[35] + h41) - 1.5 * H7;
            H34 = 3.0 * (h[31] - h[32] - h[33] + h[34]) - 3.0 * H9;
            H35 = 3.0 * (h[25] - h[26] - h[29] + h[30]) - 3.0 * H10;
        }
        // Eq. 45 without sources
        Vec<NV, R> n[16];
        n[0] = e21;
        n[1] = -0.5 * (scale(cx, F24) + scale(cy, G25) + scale(cz, H26));
        n[2] = -(1.0 / 3.0) * (scale(cx, F27) + scale(cy, G28) + scale(cz, H29));
        n[3] = e24;
        n[4] = e25;
        n[5] = e26;
        n[6] = -(scale(cx, F30) + scale(cy, 0.5 * G33) + scale(cz, 0.5 * H35));
        n[7] = -(scale(cx, 0.5 * F33) + scale(cy, G31) + scale(cz, 0.5 * H34));
        n[8] = -(scale(cx, 0.5 * F35) + scale(cy, 0.5 * G34) + scale(cz, H32));
        n[9] = -(scale(cx, 3.0 * F11) + scale(cy, G14) + scale(cz, H15));
        n[10] = -(scale(cx, F16) + scale(cy, 3.0 * G12) + scale(cz, H17));
        n[11] = -(scale(cx, F18) + scale(cy, G19) + scale(cz, 3.0 * H13));
        n[12] = -(scale(cx, 2.0 * F14) + scale(cy, 2.0 * G16) + scale(cz, H20));
        n[13] = -(scale(cx, F20) + scale(cy, 2.0 * G17) + scale(cz, 2.0 * H19));
        n[14] = -(scale(cx, 2.0 * F15) + scale(cy, G20) + scale(cz, 2.0 * H18));
        if constexpr (SRC) {        // Eq. 45, source terms
            Vec<NV, R> T[15];
            time_source_modes(w, T);
            n[0] += S1 + (8.0 / 70.0) * T[2];
            n[1] += 0.5 * T[0] - (3.0 / 7.0) * T[2];
            n[2] += T[1] / 3.0 + (4.0 / 7.0) * T[2];
            n[3] += S2 - 0.3 * T[6];
            n[4] += S3 - 0.3 * T[7];
            n[5] += S4 - 0.3 * T[8];
            n[6] += 0.5 * T[3] + 0.6 * T[6];
            n[7] += 0.5 * T[4] + 0.6 * T[7];
            n[8] += 0.5 * T[5] + 0.6 * T[8];
            n[9] += S5 + (2.0 / 3.0) * T[9];
            n[10] += S6 + (2.0 / 3.0) * T[10];
            n[11] += S7 + (2.0 / 3.0) * T[11];
            n[12] += S8 + (2.0 / 3.0) * T[12];
            n[13] += S9 + (2.0 / 3.0) * T[13];
            n[14] += S10 + (2.0 / 3.0) * T[14];
        }
        R change = R(0);
#pragma unroll
        for (int k = 0; k < 15; ++k) {
            if (conv) change = fmax(change, max_abs_diff(n[k], m[21 + k]));
            m[21 + k] = n[k];
        }
        ++ctl.iters;
        if (conv && change < R(ctl.tol) * ref) {
            ctl.capped = false;
            break;
        }
    }
    if constexpr (SRC) {            // Eq. 53 from the source at the final iterate (times dt)
        Vec<NV, R> w[43], T[15];
        build_w(w);
        time_source_modes(w, T);
        *sdt = S1 + 0.5 * T[0] + T[1] / 3.0 + 0.25 * T[2];
    }
}

template <int NV, class R>
ADER_DEV void predict_modal_src(Vec<NV, R>* m, R gm1, R cx, R cy, R cz, PredCtl& ctl, const Src<R>& src,
                                Vec<NV, R>& sdt) {
    predict_modal<NV, R, true>(m, gm1, cx, cy, cz, ctl, &src, &sdt);
}

// ------------------------------------------------------------------ nodal, App. C
// Eq. C.5 (the u35 line with node 26, the zeta node at tau = 1/3; garble G14)
template <int NV, class R>
ADER_DEV void nodal_o4_to_modes(const Vec<NV, R>* u, const Vec<NV, R>* e, Vec<NV, R>* m) {
    const Vec<NV, R>* U = u;
#define UB(n) ((n) <= 20 ? U[(n)] : e[(n) - 21])
    m[21] = 0.5 * (-5.0 * UB(1) - UB(3) - UB(4) - UB(5) - UB(6) - UB(7) - UB(8) + 12.0 * UB(21) + UB(22) + UB(23) +
                   UB(24) + UB(25) + UB(26) + UB(27) - 9.0 * UB(31) + 2.0 * UB(35));
    m[22] = 4.5 * (2.0 * UB(1) - 5.0 * UB(21) + 4.0 * UB(31) - UB(35));
    m[23] = -4.5 * (UB(1) - 3.0 * UB(21) + 3.0 * UB(31) - UB(35));
    m[24] = 3.0 * (UB(1) - 2.0 * UB(3) + UB(4) - 2.0 * UB(21) + 3.0 * UB(22) - UB(23) + UB(31) - UB(32));
    m[25] = 3.0 * (UB(1) - 2.0 * UB(5) + UB(6) - 2.0 * UB(21) + 3.0 * UB(24) - UB(25) + UB(31) - UB(33));
    m[26] = 3.0 * (UB(1) - 2.0 * UB(7) + UB(8) - 2.0 * UB(21) + 3.0 * UB(26) - UB(27) + UB(31) - UB(34));
    m[27] = -9.0 * (UB(1) - UB(3) - 2.0 * UB(21) + 2.0 * UB(22) + UB(31) - UB(32));
    m[28] = -9.0 * (UB(1) - UB(5) - 2.0 * UB(21) + 2.0 * UB(24) + UB(31) - UB(33));
    m[29] = -9.0 * (UB(1) - UB(7) - 2.0 * UB(21) + 2.0 * UB(26) + UB(31) - UB(34));
    m[30] = 6.0 * (2.0 * UB(1) - UB(3) - UB(4) - 2.0 * UB(21) + UB(22) + UB(23));
    m[31] = 6.0 * (2.0 * UB(1) - UB(5) - UB(6) - 2.0 * UB(21) + UB(24) + UB(25));
    m[32] = 6.0 * (2.0 * UB(1) - UB(7) - UB(8) - 2.0 * UB(21) + UB(26) + UB(27));
    m[33] = -12.0 * (UB(1) - UB(3) - UB(5) + UB(13) - UB(21) + UB(22) + UB(24) - UB(30));
    m[34] = -12.0 * (UB(1) - UB(5) - UB(7) + UB(9) - UB(21) + UB(24) + UB(26) - UB(28));
    m[35] = -12.0 * (UB(1) - UB(3) - UB(7) + UB(11) - UB(21) + UB(22) + UB(26) - UB(29));
#undef UB
}

// SRC: with a non-stiff source (s = dt S at nodes 1..20 once and at the tau > 0 nodes of the current
// iterate; the source terms of Eqs. C.2-C.3); sdt receives dt S-bar of Eq. C.6 from the final iterate.
template <int NV, class R, bool SRC = false>
ADER_DEV void predict_nodal(Vec<NV, R>* m, R gm1, R cx, R cy, R cz, PredCtl& ctl, const Src<R>* src = nullptr,
                            Vec<NV, R>* sdt = nullptr) {
    // Eq. C.4: the twenty tau = 0 nodes of Eq. C.1
    Vec<NV, R> u[21];
    const Vec<NV, R> q1 = 0.25 * m[2] - 0.125 * (m[8] + m[10]) + (-21.0 * m[11] + 40.0 * m[16] + 40.0 * m[18] + 60.0 * m[20]) / 960.0;
    const Vec<NV, R> q2 = 0.25 * m[3] - 0.125 * (m[8] + m[9]) + (-21.0 * m[12] + 40.0 * m[14] + 40.0 * m[19] + 60.0 * m[20]) / 960.0;
    const Vec<NV, R> q3 = 0.25 * m[4] - 0.125 * (m[9] + m[10]) + (-21.0 * m[13] + 40.0 * m[15] + 40.0 * m[17] + 60.0 * m[20]) / 960.0;
    u[1] = m[1] - (m[5] + m[6] + m[7]) / 12.0;
    u[3] = u[1] + 0.5 * m[2] + 0.25 * m[5] + 0.05 * m[11] - (m[16] + m[18]) / 24.0;
    u[4] = 2.0 * u[1] - u[3] + 0.5 * m[5];
    u[5] = u[1] + 0.5 * m[3] + 0.25 * m[6] + 0.05 * m[12] - (m[14] + m[19]) / 24.0;
    u[6] = 2.0 * u[1] - u[5] + 0.5 * m[6];
    u[7] = u[1] + 0.5 * m[4] + 0.25 * m[7] + 0.05 * m[13] - (m[15] + m[17]) / 24.0;
    u[8] = 2.0 * u[1] - u[7] + 0.5 * m[7];
    u[9] = u[5] + u[7] - u[1] + 0.25 * m[9] + 0.125 * (m[17] + m[19]);
    u[11] = u[3] + u[7] - u[1] + 0.25 * m[10] + 0.125 * (m[15] + m[18]);
    u[13] = u[3] + u[5] - u[1] + 0.25 * m[8] + 0.125 * (m[14] + m[16]);
    u[10] = 2.0 * u[7] - u[11] + 0.5 * m[5] + 0.25 * m[15];
    u[12] = 2.0 * u[3] - u[13] + 0.5 * m[6] + 0.25 * m[16];
    u[14] = 2.0 * u[5] - u[9] + 0.5 * m[7] + 0.25 * m[19];
    u[2] = u[11] + u[9] - u[7] + 0.25 * m[8] + 0.125 * (m[14] + m[16] + m[20]);
    u[15] = 2.0 * u[8] - u[14] - q1 + 0.0625 * m[5] + 0.5 * m[6] - 0.03125 * (m[14] + m[15]) - 0.25 * m[17];
    u[17] = 2.0 * u[4] - u[10] - q2 + 0.0625 * m[6] + 0.5 * m[7] - 0.03125 * (m[16] + m[17]) - 0.25 * m[18];
    u[19] = 2.0 * u[6] - u[12] - q3 + 0.5 * m[5] + 0.0625 * m[7] - 0.25 * m[14] - 0.03125 * (m[18] + m[19]);
    u[16] = u[15] + 2.0 * q1;
    u[18] = u[17] + 2.0 * q2;
    u[20] = u[19] + 2.0 * q3;
    // Eq. C.2 without sources: q-terms of the tau = 0 fluxes
    Vec<NV, R> qt[16];
    {
        Vec<NV, R> f[21], g[21], h[21];
#pragma unroll
        for (int n = 1; n <= 20; ++n) {
            const Prim<NV, R> q = primitives(u[n], gm1);
            f[n] = scale(cx, flux_from<0>(u[n], q));
            g[n] = scale(cy, flux_from<1>(u[n], q));
            h[n] = scale(cz, flux_from<2>(u[n], q));
        }
        nodal_o4_qterms(u, f, g, h, qt);
    }
    Vec<NV, R> s0[21];              // with a source: s at the tau = 0 nodes, built once
    if constexpr (SRC) {
#pragma unroll
        for (int n = 1; n <= 20; ++n) s0[n] = source_at(u[n], *src);
        nodal_o4_qterms_src(s0, qt);
    }
    // initial guess: the evolutionary modes in m[21..35] (zero: no time evolution) at the
    // tau > 0 nodes of Eq. C.1
    Vec<NV, R> e[16];
    nodal_o4_initial(u, m, e);
    const bool conv = positive_arg(ctl.tol);
    const int cap = conv ? ctl.max_iter : ctl.n_iter;
    const R ref = max_abs(m[1]) + R(sizeof(R) == 8 ? 1e-300 : 1e-30);   // never zero in R
    ctl.iters = 0;
    ctl.capped = conv;
    for (int it = 0; it < cap; ++it) {
        Vec<NV, R> f[15], g[15], h[15];          // index k - 21 for nodes 21..34
#pragma unroll
        for (int k = 0; k < 14; ++k) {
            const Prim<NV, R> q = primitives(e[k], gm1);
            f[k] = scale(cx, flux_from<0>(e[k], q));
            g[k] = scale(cy, flux_from<1>(e[k], q));
            h[k] = scale(cz, flux_from<2>(e[k], q));
        }
        Vec<NV, R> se[15];
        if constexpr (SRC) {
#pragma unroll
            for (int k = 0; k < 15; ++k) se[k] = source_at(e[k], *src);
        }
        nodal_o4_update(qt, f, g, h, e);   // Eq. C.3
        if constexpr (SRC) nodal_o4_update_src(se, e);
        ++ctl.iters;
        if (conv) {
            Vec<NV, R> old[15];
#pragma unroll
            for (int k = 0; k < 15; ++k) old[k] = m[21 + k];
            nodal_o4_to_modes(u, e, m);
            R change = R(0);
#pragma unroll
            for (int k = 0; k < 15; ++k) change = fmax(change, max_abs_diff(old[k], m[21 + k]));
            if (change < R(ctl.tol) * ref) {
                ctl.capped = false;
                break;
            }
        }
    }
    if (!conv) nodal_o4_to_modes(u, e, m);
    if constexpr (SRC) {            // Eq. C.6 from the source at the final iterate (times dt)
        Vec<NV, R> se[15];
#pragma unroll
        for (int k = 0; k < 15; ++k) se[k] = source_at(e[k], *src);
        *sdt = nodal_o4_sbar(s0, se);
    }
}

template <int NV, class R>
ADER_DEV void predict_nodal_src(Vec<NV, R>* m, R gm1, R cx, R cy, R cz, PredCtl& ctl, const Src<R>& src,
                                Vec<NV, R>& sdt) {
    predict_nodal<NV, R, true>(m, gm1, cx, cy, cz, ctl, &src, &sdt);
}



// ------------------------------------------------------------------ x+ face, Sec. V.3 and App. D
// Eqs. 64-65 for u_b and <u>; Eq. D.13 for the facial nodes; composing
// Eq. D.14 with D.15, <F> = (11 F1 - 2 (F2 + F5 + F6 + F9) - 3 F14
// + 3 (F15 + F16 + F17 + F18) + 9 F19 + 3 F24) / 24 over the nodes of Eq. D.11.
template <int D, int NV, class R>
ADER_DEV void face(const Vec<NV, R>* p, R gm1, Vec<NV, R>& ub, Vec<NV, R>& avg, Vec<NV, R>& Fa) {
    const Vec<NV, R> c1 = p[1] + 0.5 * p[21] + 0.25 * p[22] + 0.125 * p[23] +
                    (4.0 * p[5] - 2.0 * p[6] - 2.0 * p[7] + 2.0 * p[30] - p[31] - p[32]) / 24.0;
    const Vec<NV, R> c2 = 0.5 * p[2] + 0.05 * p[11] + 0.25 * p[24] + 0.125 * p[27] - (p[16] + p[18]) / 24.0;
    ub = c1 + c2;
    avg = ub + (2.0 * p[6] + 2.0 * p[7] + p[16] + p[18] + 2.0 * p[22] + 3.0 * p[23] + p[27] + p[31] + p[32]) / 24.0;
    // Eq. D.13 (caret terms of spatial modes read as w, G6)
    const Vec<NV, R> t1 = p[1] + 0.5 * p[2] + 0.05 * p[11] + (4.0 * p[5] - 2.0 * p[6] - 2.0 * p[7] - p[16] - p[18]) / 24.0;
    const Vec<NV, R> t2 = t1 + 0.5 * p[3] + 0.25 * (p[6] + p[8]) + 0.05 * p[12] + 0.125 * p[16] +
                    (0.25 * p[14] - 0.125 * p[19]) / 3.0;
    const Vec<NV, R> t3 = 0.5 * (t1 + t2) - 0.0625 * p[6] - 0.046875 * p[12] - 0.03125 * p[16];
    const Vec<NV, R> t5 = 6.0 * t1 + 3.0 * t2 - 8.0 * t3 - 0.375 * p[12];
    const Vec<NV, R> t6 = t1 + 0.5 * p[4] + 0.25 * (p[7] + p[10]) + 0.05 * p[13] + 0.125 * p[18] +
                    (0.25 * p[15] - 0.125 * p[17]) / 3.0;
    const Vec<NV, R> t7 = 0.5 * (t1 + t6) - 0.0625 * p[7] - 0.046875 * p[13] - 0.03125 * p[18];
    const Vec<NV, R> t9 = 6.0 * t1 + 3.0 * t6 - 8.0 * t7 - 0.375 * p[13];
    const Vec<NV, R> t10 = t2 + t6 - t1 + 0.25 * p[9] + 0.125 * (p[17] + p[19] + p[20]);
    const Vec<NV, R> t11 = t10 + t5 - t2 - 0.5 * p[9] - 0.25 * (p[19] + p[20]);
    const Vec<NV, R> t12 = t10 + t9 - t6 - 0.5 * p[9] - 0.25 * (p[17] + p[20]);
    const Vec<NV, R> t14 = t1 - (p[31] + p[32]) / 36.0 + (9.0 * p[21] + 3.0 * p[22] + p[23]) / 27.0 + p[24] / 6.0 +
                     (p[27] + p[30]) / 18.0;
    const Vec<NV, R> t15 = t14 + t10 - t1 +
                     (6.0 * p[25] + 6.0 * p[26] + 2.0 * p[28] + 2.0 * p[29] + 3.0 * p[31] + 3.0 * p[32] +
                      3.0 * p[33] + 3.0 * p[34] + 3.0 * p[35]) / 36.0;
    const Vec<NV, R> t16 = t15 + t11 - t10 - (6.0 * p[25] + 2.0 * p[28] + 3.0 * p[33] + 3.0 * p[34]) / 18.0;
    const Vec<NV, R> t17 = t15 + t12 - t10 - (6.0 * p[26] + 2.0 * p[29] + 3.0 * p[34] + 3.0 * p[35]) / 18.0;
    const Vec<NV, R> t18 = t16 + t17 - t15 + p[9] + 0.5 * p[20] + p[34] / 3.0;
    const Vec<NV, R> t19 = 2.0 * t14 - t1 + (2.0 * p[22] + 2.0 * p[23] + p[27]) / 9.0;
    const Vec<NV, R> t24 = t1 - 3.0 * t14 + 3.0 * t19 + 2.0 * p[23] / 9.0;
    Fa = (11.0 * flux<D>(t1, gm1) - 2.0 * (flux<D>(t2, gm1) + flux<D>(t5, gm1) + flux<D>(t6, gm1) + flux<D>(t9, gm1)) -
          3.0 * flux<D>(t14, gm1) +
          3.0 * (flux<D>(t15, gm1) + flux<D>(t16, gm1) + flux<D>(t17, gm1) + flux<D>(t18, gm1)) +
          9.0 * flux<D>(t19, gm1) + 3.0 * flux<D>(t24, gm1)) / 24.0;
}

// MHD face: all 24 facial nodes of Eq. D.11 (Eq. D.13); edge averages by
// Eq. 66 (<u>) and Eqs. D.14-D.15 (<F>) for the field component of each edge's
// EMF (slots t1+, t1-, t2+, t2-; component 5 + t1 / 5 + t2).
template <int D, class R>
ADER_DEV void face_mhd(const Vec<8, R>* p, R gm1, Vec<8, R>& ub, Vec<8, R>& avg, Vec<8, R>& Fa, R* eu, R* ef) {
    constexpr int T1 = D == 0 ? 1 : 0, T2 = D == 2 ? 1 : 2;
    const Vec<8, R> c1 = p[1] + 0.5 * p[21] + 0.25 * p[22] + 0.125 * p[23] +
                         (4.0 * p[5] - 2.0 * p[6] - 2.0 * p[7] + 2.0 * p[30] - p[31] - p[32]) / 24.0;
    const Vec<8, R> c2 = 0.5 * p[2] + 0.05 * p[11] + 0.25 * p[24] + 0.125 * p[27] - (p[16] + p[18]) / 24.0;
    ub = c1 + c2;
    avg = ub + (2.0 * p[6] + 2.0 * p[7] + p[16] + p[18] + 2.0 * p[22] + 3.0 * p[23] + p[27] + p[31] + p[32]) / 24.0;
    Vec<8, R> t[25];
    t[1] = p[1] + 0.5 * p[2] + 0.05 * p[11] + (4.0 * p[5] - 2.0 * p[6] - 2.0 * p[7] - p[16] - p[18]) / 24.0;
    t[2] = t[1] + 0.5 * p[3] + 0.25 * (p[6] + p[8]) + 0.05 * p[12] + 0.125 * p[16] + (0.25 * p[14] - 0.125 * p[19]) / 3.0;
    t[3] = 0.5 * (t[1] + t[2]) - 0.0625 * p[6] - 0.046875 * p[12] - 0.03125 * p[16];
    t[4] = 3.0 * t[1] + t[2] - 3.0 * t[3] - 0.09375 * p[12];
    t[5] = 6.0 * t[1] + 3.0 * t[2] - 8.0 * t[3] - 0.375 * p[12];
    t[6] = t[1] + 0.5 * p[4] + 0.25 * (p[7] + p[10]) + 0.05 * p[13] + 0.125 * p[18] + (0.25 * p[15] - 0.125 * p[17]) / 3.0;
    t[7] = 0.5 * (t[1] + t[6]) - 0.0625 * p[7] - 0.046875 * p[13] - 0.03125 * p[18];
    t[8] = 3.0 * t[1] + t[6] - 3.0 * t[7] - 0.09375 * p[13];
    t[9] = 6.0 * t[1] + 3.0 * t[6] - 8.0 * t[7] - 0.375 * p[13];
    t[10] = t[2] + t[6] - t[1] + 0.25 * p[9] + 0.125 * (p[17] + p[19] + p[20]);
    t[11] = t[10] + t[5] - t[2] - 0.5 * p[9] - 0.25 * (p[19] + p[20]);
    t[12] = t[10] + t[9] - t[6] - 0.5 * p[9] - 0.25 * (p[17] + p[20]);
    t[13] = t[11] + t[12] - t[10] + p[9] + 0.5 * p[20];
    t[14] = t[1] - (p[31] + p[32]) / 36.0 + (9.0 * p[21] + 3.0 * p[22] + p[23]) / 27.0 + p[24] / 6.0 + (p[27] + p[30]) / 18.0;
    t[15] = t[14] + t[10] - t[1] + (6.0 * p[25] + 6.0 * p[26] + 2.0 * p[28] + 2.0 * p[29] + 3.0 * p[31] + 3.0 * p[32] +
                                    3.0 * p[33] + 3.0 * p[34] + 3.0 * p[35]) / 36.0;
    t[16] = t[15] + t[11] - t[10] - (6.0 * p[25] + 2.0 * p[28] + 3.0 * p[33] + 3.0 * p[34]) / 18.0;
    t[17] = t[15] + t[12] - t[10] - (6.0 * p[26] + 2.0 * p[29] + 3.0 * p[34] + 3.0 * p[35]) / 18.0;
    t[18] = t[16] + t[17] - t[15] + p[9] + 0.5 * p[20] + p[34] / 3.0;
    t[19] = 2.0 * t[14] - t[1] + (2.0 * p[22] + 2.0 * p[23] + p[27]) / 9.0;
    t[20] = t[19] + t[2] - t[1] + (6.0 * p[25] + 4.0 * p[28] + 3.0 * p[31] + 3.0 * p[33]) / 18.0;
    t[21] = 2.0 * t[19] - t[20] + 0.5 * p[6] + 0.25 * p[16] + p[31] / 3.0;
    t[22] = t[19] + t[6] - t[1] + (6.0 * p[26] + 4.0 * p[29] + 3.0 * p[32] + 3.0 * p[35]) / 18.0;
    t[23] = 2.0 * t[19] - t[22] + 0.5 * p[7] + 0.25 * p[18] + p[32] / 3.0;
    t[24] = t[1] - 3.0 * t[14] + 3.0 * t[19] + 2.0 * p[23] / 9.0;
    Vec<8, R> F[25];
#pragma unroll
    for (int n = 1; n <= 24; ++n) F[n] = flux<D>(t[n], gm1);
    Fa = (11.0 * F[1] - 2.0 * (F[2] + F[5] + F[6] + F[9]) - 3.0 * F[14] + 3.0 * (F[15] + F[16] + F[17] + F[18]) +
          9.0 * F[19] + 3.0 * F[24]) / 24.0;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const int c = 5 + (s == 0 ? T1 : T2);
        auto f = [&](int n) { return F[n][c]; };
        // Eq. D.14 (the modes the edge averages need)
        const R q1 = R(3) * (f(20) - f(21)) - R(1.5) * (f(15) - f(16) + f(17) - f(18));
        const R q2 = R(1.5) * (f(20) - f(21) - f(2) + f(5));
        const R q3 = R(3) * (f(22) - f(23)) - R(1.5) * (f(15) + f(16) - f(17) - f(18));
        const R q4 = R(1.5) * (f(22) - f(23) - f(6) + f(9));
        const R m1 = (R(2) * f(1) + f(2) + f(5) + f(6) + f(9)) * R(1.0 / 6.0);
        const R m4 = R(2) * (f(2) - R(2) * f(1) + f(5));
        const R m5 = R(2) * (f(6) - R(2) * f(1) + f(9));
        const R m7 = R(16.0 / 3.0) * (f(2) - R(2) * f(3) + R(2) * f(4) - f(5));
        const R m8 = R(16.0 / 3.0) * (f(6) - R(2) * f(7) + R(2) * f(8) - f(9));
        const R m9 = R(2) * (f(10) - R(2) * f(6) + f(11) - f(12) + R(2) * f(9) - f(13));
        const R m10 = R(2) * (f(10) - R(2) * f(2) + f(12) - f(11) + R(2) * f(5) - f(13));
        const R m2 = f(2) - f(5) + m10 * R(1.0 / 12.0) - R(0.1) * m7;
        const R m3 = f(6) - f(9) + m9 * R(1.0 / 12.0) - R(0.1) * m8;
        const R m13 = R(4.5) * (f(24) - f(1)) - R(13.5) * (f(19) - f(14));
        const R m12 = R(2.25) * (f(24) - f(19) - f(14) + f(1) - R(2.0 / 3.0) * m13);
        const R m11 = R(1.5) * f(24) - R(2.5) * f(14) + R(0.25) * (f(15) + f(16) + f(17) + f(18)) - R(0.25) * m4 -
                      R(0.25) * m5 - R(4.0 / 3.0) * m12 - R(13.0 / 9.0) * m13;
        const R m14 = R(3) * q2 - R(2) * q1 - R(1.5) * m10;
        const R m16 = R(3) * (q1 - q2) + R(2.25) * m10;
        const R m15 = R(3) * q4 - R(2) * q3 - R(1.5) * m9;
        const R m17 = R(3) * (q3 - q4) + R(2.25) * m9;
        const R m18 = R(3) * (f(20) - R(2) * f(19) + f(21)) - R(1.5) * m4;
        const R m19 = R(3) * (f(22) - R(2) * f(19) + f(23)) - R(1.5) * m5;
        // Eq. D.15
        const R af = m1 + R(0.5) * m11 + m12 * R(1.0 / 3.0) + R(0.25) * m13;
        const R qa = s == 0 ? af + (R(2) * m4 + m18) * R(1.0 / 12.0) : af + (R(2) * m5 + m19) * R(1.0 / 12.0);
        const R qb = s == 0 ? R(0.5) * m2 + R(0.05) * m7 + R(0.25) * m14 + m16 * R(1.0 / 6.0)
                            : R(0.5) * m3 + R(0.05) * m8 + R(0.25) * m15 + m17 * R(1.0 / 6.0);
        ef[2 * s] = qa + qb;
        ef[2 * s + 1] = qa - qb;
        // Eq. 66
        const R qu = s == 0 ? p[3][c] + R(0.5) * (p[8][c] + p[25][c]) + R(0.25) * p[33][c] + R(0.1) * p[12][c] +
                                  (p[14][c] + R(2) * p[28][c]) * R(1.0 / 6.0)
                            : p[4][c] + R(0.5) * (p[10][c] + p[26][c]) + R(0.25) * p[35][c] + R(0.1) * p[13][c] +
                                  (p[15][c] + R(2) * p[29][c]) * R(1.0 / 6.0);
        const R up = avg[c] + (s == 0 ? (R(2) * p[6][c] + p[16][c] + p[31][c]) : (R(2) * p[7][c] + p[18][c] + p[32][c])) *
                                  R(1.0 / 12.0) + R(0.5) * qu;
        eu[2 * s] = up;
        eu[2 * s + 1] = up - qu;
    }
}

// Full edge-averaged states (all eight components; Eq. 66) for the
// linearized edge fluxes.  Slots as in face_mhd.
template <int D, class R>
ADER_DEV void edge_states(const Vec<8, R>* p, const Vec<8, R>& ub, const Vec<8, R>& avg, Vec<8, R>* e) {
    (void)ub;
    const Vec<8, R> q1 = p[3] + 0.5 * (p[8] + p[25]) + 0.25 * p[33] + 0.1 * p[12] + (p[14] + 2.0 * p[28]) / 6.0;
    const Vec<8, R> q2 = p[4] + 0.5 * (p[10] + p[26]) + 0.25 * p[35] + 0.1 * p[13] + (p[15] + 2.0 * p[29]) / 6.0;
    const Vec<8, R> u1 = avg + (2.0 * p[6] + p[16] + p[31]) / 12.0 + 0.5 * q1;
    const Vec<8, R> u2 = avg + (2.0 * p[7] + p[18] + p[32]) / 12.0 + 0.5 * q2;
    e[0] = u1;
    e[1] = u1 - q1;
    e[2] = u2;
    e[3] = u2 - q2;
}

constexpr bool HAS_SOURCE = true;
constexpr bool HAS_SOURCE_MODAL = true;

// No paired-face form at this order: the faces are evaluated one at a time.
constexpr bool HAS_FACE_PAIR = false;
template <int D, int NV, class R>
ADER_DEV void face_pair(const Vec<NV, R>*, R, Vec<NV, R>*, Vec<NV, R>*, Vec<NV, R>*) {}

}  // namespace o4
}  // namespace ader
