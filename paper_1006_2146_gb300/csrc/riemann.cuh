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
//   with |A| = R |Lambda| L of the Euler Jacobian at the arithmetic mean of
//   the two barycentre states' primitive variables.
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

// Euler only (the MHD eigen-structure is not built)
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

template <int SOLVER, int D, int NV, class R>
ADER_DEV Vec<NV, R> riemann(const FaceSide<NV, R>& L, const FaceSide<NV, R>& Rt, R gamma, R gm1) {
    if constexpr (SOLVER == 0 || NV != 5)
        return riemann_hll<D>(L, Rt, gamma, gm1);
    else
        return riemann_linearized<D>(L, Rt, gamma, gm1);
}

}  // namespace ader
