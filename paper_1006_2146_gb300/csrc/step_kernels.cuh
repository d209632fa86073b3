// The per-zone predictor + face kernel and the flux + update kernel of one
// ADER step (Sec. II: reconstruction -> space-time predictor -> face fluxes ->
// Eq. 6).  Included by the per-order translation units step_o2/3/4.cu.
//
// S3 layout: S3[((side*3 + q)*5 + v)*N + zone], side = 2*D + (S < 0),
// q = 0: barycentre state u_b (Eq. 54), 1: face average <u> (Eq. 55),
// 2: face average of the physical flux <F> (App. D).
#pragma once
#include "common.cuh"
#include "kernels.cuh"
#include "modes.cuh"
#include "riemann.cuh"

namespace ader {

template <int ORDER> struct ZoneOps;

template <int ORDER, class R>
ADER_DEV void load_modes(const StepArgs& a, const double* __restrict__ U, long long z, Vec<5, R>* m) {
    const long long N = a.grid.n;
    const R* S1 = (const R*)a.S1;
    const R* S2 = (const R*)a.S2;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        m[1][v] = R(U[v * N + z]);
#pragma unroll
        for (int d = 0; d < 3; ++d) m[2 + d][v] = S1[((0 * 3 + d) * 5 + v) * N + z];          // w2 w3 w4
        if (ORDER >= 3) {
#pragma unroll
            for (int d = 0; d < 3; ++d) m[5 + d][v] = S1[((1 * 3 + d) * 5 + v) * N + z];      // w5 w6 w7
#pragma unroll
            for (int c = 0; c < 3; ++c) m[8 + c][v] = S2[(c * 5 + v) * N + z];                 // w8 w9 w10
        }
        if (ORDER == 4) {
#pragma unroll
            for (int d = 0; d < 3; ++d) m[11 + d][v] = S1[((2 * 3 + d) * 5 + v) * N + z];     // w11 w12 w13
#pragma unroll
            for (int c = 0; c < 7; ++c) m[14 + c][v] = S2[((3 + c) * 5 + v) * N + z];          // w14..w20
        }
    }
}

template <int ORDER, int D, int S, class R>
ADER_DEV void store_face(const StepArgs& a, long long z, const Vec<5, R>* m, R gm1) {
    constexpr int L = ModeCount<ORDER>::L;
    Vec<5, R> p[L + 1];
    to_face_frame<ORDER, D, S>(m, p);
    Vec<5, R> ub, avg, Fa;
    ZoneOps<ORDER>::template face<D>(p, gm1, ub, avg, Fa);
    // a non-physical barycentre state is replaced by the zone average for the wave speeds
    const Prim<R> q = primitives(ub, gm1);
    if (!(ub[0] > R(0)) || !(q.p > R(0))) ub = m[1];
    constexpr int side = 2 * D + (S < 0 ? 1 : 0);
    R* S3 = (R*)a.S3;
    const long long N = a.grid.n;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        S3[((side * 3 + 0) * 5 + v) * N + z] = ub[v];
        S3[((side * 3 + 1) * 5 + v) * N + z] = avg[v];
        S3[((side * 3 + 2) * 5 + v) * N + z] = Fa[v];
    }
}

template <int ORDER, int FORM, class R>
ADER_DEV void zone_predict_faces(const StepArgs& a, const double* __restrict__ U, long long z) {
    constexpr int LS = ModeCount<ORDER>::LS, L = ModeCount<ORDER>::L;
    Vec<5, R> m[L + 1];
    load_modes<ORDER>(a, U, z, m);
#pragma unroll
    for (int k = LS + 1; k <= L; ++k) m[k] = vzero<5, R>();
    const double dt = a.dt_dev ? *a.dt_dev : a.dt;
    const R gm1 = R(a.gamma - 1.0);
    const R cx = R(dt / a.dx[0]), cy = R(dt / a.dx[1]), cz = R(dt / a.dx[2]);
    if (a.n_iter > 0) {      // n_iter = 0: spatial polynomial only (SSP-RK face rule)
        if (FORM == FORM_MODAL)
            ZoneOps<ORDER>::predict_modal(m, gm1, cx, cy, cz, a.n_iter);
        else
            ZoneOps<ORDER>::predict_nodal(m, gm1, cx, cy, cz, a.n_iter);
    }
    store_face<ORDER, 0, +1>(a, z, m, gm1);
    store_face<ORDER, 0, -1>(a, z, m, gm1);
    store_face<ORDER, 1, +1>(a, z, m, gm1);
    store_face<ORDER, 1, -1>(a, z, m, gm1);
    store_face<ORDER, 2, +1>(a, z, m, gm1);
    store_face<ORDER, 2, -1>(a, z, m, gm1);
}

template <int ORDER, int FORM, class R>
__global__ void __launch_bounds__(128) k_predict_faces(StepArgs a, const double* __restrict__ U) {
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (z < a.grid.n) zone_predict_faces<ORDER, FORM, R>(a, U, z);
}

template <class R>
ADER_DEV FaceSide<R> load_side(const StepArgs& a, int side, long long z) {
    const R* S3 = (const R*)a.S3;
    const long long N = a.grid.n;
    FaceSide<R> s;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        s.ub[v] = S3[((side * 3 + 0) * 5 + v) * N + z];
        s.avg[v] = S3[((side * 3 + 1) * 5 + v) * N + z];
        s.F[v] = S3[((side * 3 + 2) * 5 + v) * N + z];
    }
    return s;
}

// F(i+1/2) - F(i-1/2) in direction D, accumulated in FP64.  The same
// function with the same operands computes a face's flux for both of its
// zones, so the two values are identical and Eq. 6 telescopes exactly.
template <int SOLVER, int D, class R>
ADER_DEV void flux_difference(const StepArgs& a, long long z, int i, int j, int k, R gamma, R gm1, double* acc) {
    const long long zp = nbr(a.grid, i, j, k, D == 0, D == 1, D == 2);
    const long long zm = nbr(a.grid, i, j, k, -(D == 0), -(D == 1), -(D == 2));
    const Vec<5, R> Fp = riemann<SOLVER, D>(load_side<R>(a, 2 * D, z), load_side<R>(a, 2 * D + 1, zp), gamma, gm1);
    const Vec<5, R> Fm = riemann<SOLVER, D>(load_side<R>(a, 2 * D, zm), load_side<R>(a, 2 * D + 1, z), gamma, gm1);
    const double inv = 1.0 / a.dx[D];
#pragma unroll
    for (int v = 0; v < 5; ++v) acc[v] -= ((double)Fp[v] - (double)Fm[v]) * inv;
}

template <int SOLVER, class R>
ADER_DEV void zone_flux_update(const StepArgs& a, double* out, const double* base, double c_host, int use_dt_dev,
                               long long z) {
    const int i = (int)(z % a.grid.nx);
    const long long t = z / a.grid.nx;
    const int j = (int)(t % a.grid.ny), k = (int)(t / a.grid.ny);
    const R gamma = R(a.gamma), gm1 = R(a.gamma - 1.0);
    double acc[5] = {0, 0, 0, 0, 0};
    flux_difference<SOLVER, 0, R>(a, z, i, j, k, gamma, gm1, acc);
    flux_difference<SOLVER, 1, R>(a, z, i, j, k, gamma, gm1, acc);
    flux_difference<SOLVER, 2, R>(a, z, i, j, k, gamma, gm1, acc);
    const double c = use_dt_dev ? c_host * (*a.dt_dev) : c_host;
    const long long N = a.grid.n;
    bool bad = false;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        const double val = (base ? base[v * N + z] : 0.0) + c * acc[v];
        bad |= !isfinite(val);
        out[v * N + z] = val;
    }
    if (bad) raise_flag(a.flag, FLAG_NONFINITE);
}

template <int SOLVER, class R>
__global__ void __launch_bounds__(128) k_flux_update(StepArgs a, double* out, const double* base, double c_host,
                                                     int use_dt_dev) {
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (z < a.grid.n) zone_flux_update<SOLVER, R>(a, out, base, c_host, use_dt_dev, z);
}

template <int ORDER, class R>
int launch_predict_faces_order(const StepArgs& a, const double* U, cudaStream_t st) {
    const int T = 128;
    const unsigned blocks = (unsigned)((a.grid.n + T - 1) / T);
    if (a.form == FORM_MODAL)
        k_predict_faces<ORDER, FORM_MODAL, R><<<blocks, T, 0, st>>>(a, U);
    else
        k_predict_faces<ORDER, FORM_NODAL, R><<<blocks, T, 0, st>>>(a, U);
    return 1;
}

}  // namespace ader
