// Space-time averaged numerical flux at a face with the eigen-structure frozen
// at the face's space-time barycentre (Sec. II.3, Eq. 56).
//
// Inputs per face i+1/2 of direction D: the left zone's + side and the right
// zone's - side, each holding the barycentre state u_b (Eq. 54, already
// replaced by the zone average when non-physical), <u> (Eq. 55) and the
// averaged physical flux <F> = dx/dt <f>.
//
// Readings (the paper is silent):
//   HLL: lambda_L = min(v_L - a_L, v_R - a_R, 0), lambda_R = max(v_L + a_L, v_R + a_R, 0).
//   Linearized (Roe / Harten-Hyman form): F = (<F>_L + <F>_R)/2 - |A| (<u>_R - <u>_L)/2
//   with |A| = R |Lambda| L of the flux Jacobian at the arithmetic mean of
//   the two barycentre states' primitive variables.  For MHD the row and
//   column of the normal field are left out (it is continuous across the
//   face and carries no flux), which leaves the seven-wave system.
#pragma once
#include "common.cuh"

namespace ader {

template <int NV, class R>
struct FaceSide {
    Vec<NV, R> ub, avg, F;
};

// HLL with the fast speeds (sound speeds for Euler) of the barycentre states
template <int D, int NV, class R>
ADER_DEV Vec<NV, R> riemann_hll(const FaceSide<NV, R>& L, const FaceSide<NV, R>& Rt, R gamma, R gm1) {
    const Prim<NV, R> pl = primitives(L.ub, gm1), pr = primitives(Rt.ub, gm1);
    const R vl = D == 0 ? pl.vx : (D == 1 ? pl.vy : pl.vz);
    const R vr = D == 0 ? pr.vx : (D == 1 ? pr.vy : pr.vz);
    const R al = fast_speed<D>(L.ub, pl, gamma), ar = fast_speed<D>(Rt.ub, pr, gamma);
    const R lamL = fmin(fmin(vl - al, vr - ar), R(0));
    const R lamR = fmax(fmax(vl + al, vr + ar), R(0));
    const R inv = rcp(lamR - lamL);
    const R wl = lamR * inv, wr = -lamL * inv, wd = lamR * lamL * inv;
    Vec<NV, R> out;
#pragma unroll
    for (int v = 0; v < NV; ++v) out[v] = wl * L.F[v] + wr * Rt.F[v] + wd * (Rt.avg[v] - L.avg[v]);
    return out;
}

// Euler: the textbook eigenvectors
template <int D, class R>
ADER_DEV Vec<5, R> riemann_linearized(const FaceSide<5, R>& L, const FaceSide<5, R>& Rt, R gamma, R gm1) {
    const Prim<5, R> pl = primitives(L.ub, gm1), pr = primitives(Rt.ub, gm1);
    const R rho = R(0.5) * (L.ub[0] + Rt.ub[0]);
    const R v[3] = {R(0.5) * (pl.vx + pr.vx), R(0.5) * (pl.vy + pr.vy), R(0.5) * (pl.vz + pr.vz)};
    const R p = R(0.5) * (pl.p + pr.p);
    const R a2 = gamma * p / rho, a = sqrt(a2);
    const R q2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    const R H = a2 / gm1 + R(0.5) * q2;
    constexpr int T1 = D == 0 ? 1 : 0, T2 = D == 2 ? 1 : 2;
    const R un = v[D], ut1 = v[T1], ut2 = v[T2];
    Vec<5, R> dU;
#pragma unroll
    for (int c = 0; c < 5; ++c) dU[c] = Rt.avg[c] - L.avg[c];
    // wave strengths: L (<u>_R - <u>_L)
    const R at1 = dU[1 + T1] - ut1 * dU[0];
    const R at2 = dU[1 + T2] - ut2 * dU[0];
    const R d5 = dU[4] - at1 * ut1 - at2 * ut2;
    const R a2s = gm1 / a2 * (dU[0] * (H - un * un) + un * dU[1 + D] - d5);
    const R a1s = (dU[0] * (un + a) - dU[1 + D] - a * a2s) / (R(2) * a);
    const R a5s = dU[0] - a1s - a2s;
    const R l1 = fabs(un - a), l2 = fabs(un), l5 = fabs(un + a);
    const R s1 = l1 * a1s, s2 = l2 * a2s, s5 = l5 * a5s, st1 = l2 * at1, st2 = l2 * at2;
    // |A| dU = sum of |lambda| alpha r over the five right eigenvectors
    Vec<5, R> diss;
    diss[0] = s1 + s2 + s5;
    diss[1 + D] = s1 * (un - a) + s2 * un + s5 * (un + a);
    diss[1 + T1] = (s1 + s2 + s5) * ut1 + st1;
    diss[1 + T2] = (s1 + s2 + s5) * ut2 + st2;
    diss[4] = s1 * (H - un * a) + s2 * R(0.5) * q2 + s5 * (H + un * a) + st1 * ut1 + st2 * ut2;
    Vec<5, R> out;
#pragma unroll
    for (int c = 0; c < 5; ++c) out[c] = R(0.5) * (L.F[c] + Rt.F[c]) - R(0.5) * diss[c];
    return out;
}

// Ideal MHD (Gaussian units): |A| dU of the seven-wave system in direction D
// at the state (rho, v, p, B).  The jump is taken to primitive variables
// W = (rho, v_n, v_t1, v_t2, p, b_t1, b_t2), b = B / sqrt(4 pi); there it is
// split into the entropy, Alfven (u -+ c_a), fast (u -+ c_f) and slow
// (u -+ c_s) waves with the eigenvectors normalised by
//   alpha_f^2 = (a^2 - c_s^2) / (c_f^2 - c_s^2),  alpha_s^2 = (c_f^2 - a^2) / (c_f^2 - c_s^2),
//   (beta_t1, beta_t2) = b_t / |b_t|  (1/sqrt 2 each when b_t = 0),
// which stay finite where the speeds coincide; each amplitude is scaled by
// its |lambda| and the sum is mapped back to conserved variables.
template <int D, class R>
ADER_DEV Vec<8, R> mhd_abs_jacobian_apply(R rho, const R* v, R p, const R* B, R gamma, R gm1, const Vec<8, R>& dU) {
    constexpr int T1 = D == 0 ? 1 : 0, T2 = D == 2 ? 1 : 2;
    const R k = R(0.28209479177387814);        // 1 / sqrt(4 pi)
    const R bx = B[D] * k, by = B[T1] * k, bz = B[T2] * k;
    const R u = v[D], vt1 = v[T1], vt2 = v[T2];
    const R irho = rcp(rho), sr = sqrt(rho), isr = rcp(sr);
    const R a2 = gamma * p * irho, a = sqrt(a2);
    const R ca2 = bx * bx * irho, bt2 = (by * by + bz * bz) * irho;
    const R sum = a2 + ca2 + bt2;
    const R disc = sqrt(fmax(sum * sum - R(4) * a2 * ca2, R(0)));
    const R cf2 = R(0.5) * (sum + disc), cs2 = fmax(R(0.5) * (sum - disc), R(0));
    const R cf = sqrt(cf2), cs = sqrt(cs2), ca = sqrt(ca2);
    const R tiny = sizeof(R) == 8 ? R(1e-12) : R(1e-6);
    const R dc = cf2 - cs2;
    R af = R(1), as = R(0);
    if (dc > tiny * cf2) {
        af = sqrt(fmax(a2 - cs2, R(0)));
        as = sqrt(fmax(cf2 - a2, R(0)));
        const R n = rcp(sqrt(af * af + as * as));       // af^2 + as^2 = 1 up to round-off
        af *= n;
        as *= n;
    }
    const R bt = sqrt(by * by + bz * bz);
    R ey = R(0.70710678118654752), ez = R(0.70710678118654752);
    if (bt > tiny * sqrt(rho * sum)) {
        ey = by / bt;
        ez = bz / bt;
    }
    const R sg = bx >= R(0) ? R(1) : R(-1);
    // primitive jump
    const R drho = dU[0];
    const R du = (dU[1 + D] - u * drho) * irho, dv = (dU[1 + T1] - vt1 * drho) * irho;
    const R dw = (dU[1 + T2] - vt2 * drho) * irho;
    const R dby = dU[5 + T1] * k, dbz = dU[5 + T2] * k;
    const R q2 = u * u + vt1 * vt1 + vt2 * vt2;
    const R dp = gm1 * (dU[4] - R(0.5) * q2 * drho - rho * (u * du + vt1 * dv + vt2 * dw) - by * dby - bz * dbz);
    // amplitudes
    const R dvpar = ey * dv + ez * dw, dvper = -ez * dv + ey * dw;
    const R dbpar = ey * dby + ez * dbz, dbper = -ez * dby + ey * dbz;
    const R Ap = R(0.5) * (dvper - sg * isr * dbper), Am = R(0.5) * (dvper + sg * isr * dbper);
    const R fc = af * cf, sc = as * cs;
    const R idet = rcp(fc * fc + sc * sc);
    const R Fd = (fc * du - sc * sg * dvpar) * idet, Sd = (sc * du + fc * sg * dvpar) * idet;
    const R X = dp * irho / a2, Y = dbpar * isr / a;
    const R Fs = af * X + as * Y, Ss = as * X - af * Y;
    const R E = drho - dp / a2;
    // scaled by |lambda|
    const R wE = fabs(u) * E;
    const R wFp = fabs(u + cf) * R(0.5) * (Fs + Fd), wFm = fabs(u - cf) * R(0.5) * (Fs - Fd);
    const R wSp = fabs(u + cs) * R(0.5) * (Ss + Sd), wSm = fabs(u - cs) * R(0.5) * (Ss - Sd);
    const R wAp = fabs(u + ca) * Ap, wAm = fabs(u - ca) * Am;
    const R Fsum = wFp + wFm, Fdif = wFp - wFm, Ssum = wSp + wSm, Sdif = wSp - wSm;
    // sum of the scaled right eigenvectors, primitive
    const R Drho = wE + rho * (af * Fsum + as * Ssum);
    const R Du = fc * Fdif + sc * Sdif;
    const R Dvpar = sg * (-sc * Fdif + fc * Sdif), Dvper = wAp + wAm;
    const R Dp = rho * a2 * (af * Fsum + as * Ssum);
    const R Dbpar = a * sr * (as * Fsum - af * Ssum), Dbper = -sg * sr * (wAp - wAm);
    const R Dv = ey * Dvpar - ez * Dvper, Dw = ez * Dvpar + ey * Dvper;
    const R Dby = ey * Dbpar - ez * Dbper, Dbz = ez * Dbpar + ey * Dbper;
    // back to conserved variables
    Vec<8, R> out;
    out[0] = Drho;
    out[1 + D] = u * Drho + rho * Du;
    out[1 + T1] = vt1 * Drho + rho * Dv;
    out[1 + T2] = vt2 * Drho + rho * Dw;
    out[4] = R(0.5) * q2 * Drho + rho * (u * Du + vt1 * Dv + vt2 * Dw) + Dp / gm1 + by * Dby + bz * Dbz;
    out[5 + D] = R(0);
    out[5 + T1] = Dby / k;
    out[5 + T2] = Dbz / k;
    return out;
}

// the arithmetic mean of the primitive variables of two states (the linearisation state)
template <class R>
struct MeanState {
    R rho, v[3], p, B[3];
};

template <class R>
ADER_DEV MeanState<R> mhd_mean_state(const Vec<8, R>& uL, const Vec<8, R>& uR, R gm1) {
    const Prim<8, R> pl = primitives(uL, gm1), pr = primitives(uR, gm1);
    MeanState<R> m;
    m.rho = R(0.5) * (uL[0] + uR[0]);
    m.v[0] = R(0.5) * (pl.vx + pr.vx);
    m.v[1] = R(0.5) * (pl.vy + pr.vy);
    m.v[2] = R(0.5) * (pl.vz + pr.vz);
    m.p = R(0.5) * (pl.p + pr.p);
#pragma unroll
    for (int c = 0; c < 3; ++c) m.B[c] = R(0.5) * (uL[5 + c] + uR[5 + c]);
    return m;
}

template <int D, class R>
ADER_DEV Vec<8, R> riemann_linearized_mhd(const FaceSide<8, R>& L, const FaceSide<8, R>& Rt, R gamma, R gm1) {
    const MeanState<R> m = mhd_mean_state(L.ub, Rt.ub, gm1);
    Vec<8, R> dU;
#pragma unroll
    for (int c = 0; c < 8; ++c) dU[c] = Rt.avg[c] - L.avg[c];
    const Vec<8, R> diss = mhd_abs_jacobian_apply<D, R>(m.rho, m.v, m.p, m.B, gamma, gm1, dU);
    Vec<8, R> out;
#pragma unroll
    for (int c = 0; c < 8; ++c) out[c] = R(0.5) * (L.F[c] + Rt.F[c]) - R(0.5) * diss[c];
    return out;
}

template <int SOLVER, int D, int NV, class R>
ADER_DEV Vec<NV, R> riemann(const FaceSide<NV, R>& L, const FaceSide<NV, R>& Rt, R gamma, R gm1) {
    if constexpr (SOLVER == 0)
        return riemann_hll<D>(L, Rt, gamma, gm1);
    else if constexpr (NV == 5)
        return riemann_linearized<D>(L, Rt, gamma, gm1);
    else
        return riemann_linearized_mhd<D>(L, Rt, gamma, gm1);
}

}  // namespace ader
