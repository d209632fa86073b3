// The per-zone predictor + face kernel, the flux + update kernel and, for
// MHD, the edge-EMF and constrained-transport kernels of one ADER step
// (Sec. II: reconstruction -> space-time predictor -> face fluxes -> Eqs. 6, 8).
// Instantiated per (order, variables, precision) through step_inst.cuh.
//
// S3 layout: S3[(side*NQ + q)*N + zone], side = 2*D + (S < 0), NQ =
// side_values(NV): q in [0, NV) barycentre state u_b (Eq. 54), [NV, 2NV) face
// average <u> (Eq. 55), [2NV, 3NV) face average of the physical flux <F>
// (App. D); MHD adds, for the four edges t1+, t1-, t2+, t2- of the face, the
// edge averages <u_c> and <F_c> (Eq. 57, Eqs. D.5/D.10/D.15) of the field
// component c = 5 + t the edge's EMF needs.
#pragma once
#include "common.cuh"
#include "kernels.cuh"
#include "modes.cuh"
#include "riemann.cuh"
#include "mlp.cuh"

namespace ader {

template <int ORDER> struct ZoneOps;

template <int ORDER, int NV, class R>
ADER_DEV void load_modes(const StepArgs& a, const double* __restrict__ U, long long z, Vec<NV, R>* m) {
    const long long N = a.grid.n;
    const R* S1 = (const R*)a.S1;
    const R* S2 = (const R*)a.S2;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        if constexpr (sizeof(R) == 4)       // FP32 bulk: the zone means from the FP32 copy of the state
            m[1][v] = v < 5 ? (a.Uf ? a.Uf[v * N + z] : R(U[v * N + z])) : ((const R*)a.ZB)[(v - 5) * N + z];
        else
            m[1][v] = v < 5 ? R(U[v * N + z]) : ((const R*)a.ZB)[(v - 5) * N + z];
#pragma unroll
        for (int d = 0; d < 3; ++d) m[2 + d][v] = S1[((0 * 3 + d) * NV + v) * N + z];          // w2 w3 w4
        if (ORDER >= 3) {
#pragma unroll
            for (int d = 0; d < 3; ++d) m[5 + d][v] = S1[((1 * 3 + d) * NV + v) * N + z];      // w5 w6 w7
#pragma unroll
            for (int c = 0; c < 3; ++c) m[8 + c][v] = S2[(c * NV + v) * N + z];                 // w8 w9 w10
        }
        if (ORDER == 4) {
#pragma unroll
            for (int d = 0; d < 3; ++d) m[11 + d][v] = S1[((2 * 3 + d) * NV + v) * N + z];     // w11 w12 w13
#pragma unroll
            for (int c = 0; c < 7; ++c) m[14 + c][v] = S2[((3 + c) * NV + v) * N + z];          // w14..w20
        }
    }
}

// the Euler part of one face side: the barycentre state (replaced by the zone
// average for the wave speeds when it is not physical), <u> and <F>
template <int D, int S, int NV, class R>
ADER_DEV void write_side(const StepArgs& a, long long z, const Vec<NV, R>& mean, Vec<NV, R> ub, const Vec<NV, R>& avg,
                         const Vec<NV, R>& Fa, R gm1) {
    constexpr int NQ = side_values(NV);
    const Prim<NV, R> q = primitives(ub, gm1);
    if (!(ub[0] > R(0)) || !(q.p > R(0))) ub = mean;
    constexpr int side = 2 * D + (S < 0 ? 1 : 0);
    R* S3 = (R*)a.S3;
    const long long N = a.grid.n;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        S3[(side * NQ + v) * N + z] = ub[v];
        S3[(side * NQ + NV + v) * N + z] = avg[v];
        S3[(side * NQ + 2 * NV + v) * N + z] = Fa[v];
    }
}

template <int ORDER, int D, int S, int NV, class R>
ADER_DEV void store_face(const StepArgs& a, long long z, const Vec<NV, R>* m, R gm1) {
    constexpr int L = ModeCount<ORDER>::L;
    constexpr int NQ = side_values(NV);
    Vec<NV, R> p[L + 1];
    to_face_frame<ORDER, D, S>(m, p);
    Vec<NV, R> ub, avg, Fa;
    R eu[4], ef[4];
    if constexpr (NV == 8)
        ZoneOps<ORDER>::template face_mhd<D>(p, gm1, ub, avg, Fa, eu, ef);
    else
        ZoneOps<ORDER>::template face<D>(p, gm1, ub, avg, Fa);
    write_side<D, S>(a, z, m[1], ub, avg, Fa, gm1);
    if constexpr (NV == 8) {
        constexpr int side = 2 * D + (S < 0 ? 1 : 0);
        R* S3 = (R*)a.S3;
        const long long N = a.grid.n;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            S3[(side * NQ + 3 * NV + 2 * e) * N + z] = eu[e];
            S3[(side * NQ + 3 * NV + 2 * e + 1) * N + z] = ef[e];
        }
        if (a.solver == SOLVER_LINEARIZED) {      // the linearized edge fluxes need every component
            Vec<8, R> es[4];
            ZoneOps<ORDER>::template edge_states<D>(p, ub, avg, es);
            R* X = S3 + (long long)6 * NQ * N;
#pragma unroll
            for (int e = 0; e < 4; ++e)
#pragma unroll
                for (int v = 0; v < 8; ++v) X[(side * EDGE_STATE_VALUES + e * 8 + v) * N + z] = es[e][v];
        }
    }
}

// both faces of direction D: the paired form where the order has one (Euler), else one face at a time
template <int ORDER, int D, int NV, class R>
ADER_DEV void store_faces(const StepArgs& a, long long z, const Vec<NV, R>* m, R gm1) {
    if constexpr (NV == 5 && ZoneOps<ORDER>::HAS_FACE_PAIR) {
        constexpr int L = ModeCount<ORDER>::L;
        Vec<NV, R> p[L + 1];
        to_face_frame<ORDER, D, +1>(m, p);
        Vec<NV, R> ub[2], avg[2], Fa[2];
        ZoneOps<ORDER>::template face_pair<D>(p, gm1, ub, avg, Fa);
        write_side<D, +1>(a, z, m[1], ub[0], avg[0], Fa[0], gm1);
        write_side<D, -1>(a, z, m[1], ub[1], avg[1], Fa[1], gm1);
    } else {
        store_face<ORDER, D, +1>(a, z, m, gm1);
        store_face<ORDER, D, -1>(a, z, m, gm1);
    }
}

// Iteration statistics of the converged predictor: sum, maximum and capped zones.
ADER_DEV void record_iterations(unsigned long long* stats, const PredCtl& ctl) {
#ifdef __CUDA_ARCH__
    // one set of atomics per warp: the counters are shared by every zone of the grid
    const unsigned mask = __activemask();
    const unsigned sum = __reduce_add_sync(mask, (unsigned)ctl.iters);
    const unsigned mx = __reduce_max_sync(mask, (unsigned)ctl.iters);
    const unsigned capped = __reduce_add_sync(mask, ctl.capped ? 1u : 0u);
    if ((threadIdx.x & 31) == __ffs(mask) - 1) {
        atomicAdd(&stats[0], (unsigned long long)sum);
        atomicMax(&stats[1], (unsigned long long)mx);
        if (capped) atomicAdd(&stats[2], (unsigned long long)capped);
    }
#else
    stats[0] += ctl.iters;
    if ((unsigned long long)ctl.iters > stats[1]) stats[1] = ctl.iters;
    if (ctl.capped) stats[2] += 1;
#endif
}

// The ADER-CG predictor of zone z (Sec. II.2): the spatial modes, the learned or zero initial guess of
// the evolutionary modes, the iteration, and what the step keeps besides the face data (dt S-bar with a
// source, the whole space-time polynomial for dense output).  m[1..L] holds the space-time modes after.
// SRC: the context carries a non-stiff source (orders with ZoneOps::HAS_SOURCE); the predictor then also
// writes dt S-bar of Eq. 6 for the update (a.Sb).
// dt_in: the step size (the caller reads a.dt_dev, once per thread where it can)
template <int ORDER, int FORM, int NV, class R, bool SRC = false>
ADER_DEV void zone_predict(const StepArgs& a, const double* __restrict__ U, long long z, Vec<NV, R>* m, R dt) {
    constexpr int LS = ModeCount<ORDER>::LS, L = ModeCount<ORDER>::L;
    load_modes<ORDER>(a, U, z, m);
#pragma unroll
    for (int k = LS + 1; k <= L; ++k) m[k] = vzero<NV, R>();
    const R gm1 = arg_gm1<R>(a);
    const R cx = dt * arg_idx<R>(a, 0), cy = dt * arg_idx<R>(a, 1), cz = dt * arg_idx<R>(a, 2);
    if (a.n_iter > 0) {      // n_iter = 0: spatial polynomial only (SSP-RK face rule)
        if constexpr (ORDER == 3) {
            if (a.G && (!a.Gact || a.Gact[z])) {          // learned initial guess of the evolutionary modes
#pragma unroll
                for (int j = 0; j < 5; ++j)
#pragma unroll
                    for (int v = 0; v < NV; ++v) m[11 + j][v] = R(a.G[(long long)(j * NV + v) * a.grid.n + z]);
            }
        }
        PredCtl ctl{a.n_iter, a.tol, a.max_iter, 0, false};
        if constexpr (SRC) {
            Src<R> src;
            src.kind = a.src_kind;
#pragma unroll
            for (int i = 0; i < 3; ++i) src.a[i] = dt * bulk_arg<R>(a.src_par[i]);
            Vec<NV, R> sdt;
            if (FORM == FORM_MODAL)
                ZoneOps<ORDER>::predict_modal_src(m, gm1, cx, cy, cz, ctl, src, sdt);
            else
                ZoneOps<ORDER>::predict_nodal_src(m, gm1, cx, cy, cz, ctl, src, sdt);
            R* Sb = (R*)a.Sb;
#pragma unroll
            for (int v = 0; v < 5; ++v) Sb[v * a.grid.n + z] = sdt[v];
        } else if (FORM == FORM_MODAL) {
            ZoneOps<ORDER>::predict_modal(m, gm1, cx, cy, cz, ctl);
        } else {
            ZoneOps<ORDER>::predict_nodal(m, gm1, cx, cy, cz, ctl);
        }
        if (a.stats && positive_arg(a.tol)) record_iterations(a.stats, ctl);
        if (ctl.capped) raise_flag(a.flag, FLAG_NOT_CONVERGED);
    }
    if (a.modes_out) {      // dense output (Sec. VII): keep the whole space-time polynomial of the step
        R* o = (R*)a.modes_out;
#pragma unroll
        for (int k = 1; k <= L; ++k)
#pragma unroll
            for (int v = 0; v < NV; ++v) o[(long long)((k - 1) * NV + v) * a.grid.n + z] = m[k][v];
    }
}

template <int ORDER, int FORM, int NV, class R, bool SRC = false>
ADER_DEV void zone_predict_faces(const StepArgs& a, const double* __restrict__ U, long long z) {
    Vec<NV, R> m[ModeCount<ORDER>::L + 1];
    zone_predict<ORDER, FORM, NV, R, SRC>(a, U, z, m, bulk_arg<R>(a.dt_dev ? *a.dt_dev : a.dt));
    const R gm1 = arg_gm1<R>(a);
    store_faces<ORDER, 0>(a, z, m, gm1);
    store_faces<ORDER, 1>(a, z, m, gm1);
    store_faces<ORDER, 2>(a, z, m, gm1);
}

// FP32 bulk asks for three 128-thread blocks per SM at orders 2-3 (at most 168 registers, a few hundred
// bytes of spills to L1): the extra warps hide more latency than the spills cost (about 12% per 256^3
// step).  At order 4, and for MHD at order 3, the predictor spills kilobytes per zone at 168 registers;
// there it takes two blocks per SM and 255 registers (a 128^3 MHD step at order 3: 3.5 -> 2.4 ms).
template <int ORDER, int FORM, int NV, class R, bool SRC = false>
__global__ void __launch_bounds__(128, sizeof(R) == 4 ? (ORDER == 4 || (ORDER == 3 && NV == 8) ? 2 : 3) : 1)
    k_predict_faces(StepArgs a, const double* __restrict__ U) {
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (z < a.grid.n) zone_predict_faces<ORDER, FORM, NV, R, SRC>(a, U, z);
}

template <int NV, class R>
ADER_DEV FaceSide<NV, R> load_side(const StepArgs& a, int side, long long z) {
    constexpr int NQ = side_values(NV);
    const R* S3 = (const R*)a.S3;
    const long long N = a.grid.n;
    FaceSide<NV, R> s;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        s.ub[v] = S3[(side * NQ + v) * N + z];
        s.avg[v] = S3[(side * NQ + NV + v) * N + z];
        s.F[v] = S3[(side * NQ + 2 * NV + v) * N + z];
    }
    return s;
}

// Eq. 6 for zone z: out = base + c sum_D (F(i_D - 1/2) - F(i_D + 1/2)) / dx_D,
// accumulated in FP64 for the five hydrodynamic variables.  Two ways to the
// same fluxes:
//  * fused (zone_flux_update): each zone solves the two faces of each
//    direction itself -- every face twice over the grid, in one pass.  The
//    same function with the same operands gives both zones of a face the same
//    value, so Eq. 6 telescopes exactly.  Used by the FP32-bulk kernels, whose
//    cost there is the FP64 accumulation, not the Riemann solves.
//  * stored (zone_face_fluxes, then zone_flux_update_stored): every face is
//    solved once, by the zone below it, into the WENO scratch S1 (dead once
//    the face data exist; at least 15 values per zone at every order), and
//    the update takes differences of stored values.  Used by FP64, where the
//    solves are FP64 work on the critical path.
template <int SOLVER, int D, int NV, class R>
ADER_DEV Vec<NV, R> upper_face_flux(const StepArgs& a, long long z, int i, int j, int k, R gamma, R gm1) {
    const long long zp = nbr_along(a.grid, z, i, j, k, D, 1);
    return riemann<SOLVER, D>(load_side<NV, R>(a, 2 * D, z), load_side<NV, R>(a, 2 * D + 1, zp), gamma, gm1);
}

template <int SOLVER, int D, int NV, class R>
ADER_DEV void flux_difference(const StepArgs& a, long long z, int i, int j, int k, R gamma, R gm1, double* acc) {
    const long long zm = nbr_along(a.grid, z, i, j, k, D, -1);
    const Vec<NV, R> Fp = upper_face_flux<SOLVER, D, NV, R>(a, z, i, j, k, gamma, gm1);
    const Vec<NV, R> Fm = riemann<SOLVER, D>(load_side<NV, R>(a, 2 * D, zm), load_side<NV, R>(a, 2 * D + 1, z),
                                             gamma, gm1);
    const double inv = a.idx[D];
#pragma unroll
    for (int v = 0; v < 5; ++v) acc[v] -= ((double)Fp[v] - (double)Fm[v]) * inv;
}

// out = base + c acc (+ dt S-bar of Eq. 6 where the predictor wrote one, a.Sb in the bulk precision R)
template <class R>
ADER_DEV void store_update(const StepArgs& a, double* out, const double* base, double c_host, int use_dt_dev,
                           const double* acc, long long z) {
    const double c = use_dt_dev ? c_host * (*a.dt_dev) : c_host;
    const long long N = a.grid.n;
    const R* Sb = (const R*)a.Sb;
    bool bad = false;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        double val = (base ? base[v * N + z] : 0.0) + c * acc[v];
        if (Sb) val += (double)Sb[v * N + z];
        bad |= !isfinite(val);
        out[v * N + z] = val;
    }
    if (bad && !a.defer_nonfinite) raise_flag(a.flag, FLAG_NONFINITE);
}

template <int SOLVER, int NV, class R>
ADER_DEV void zone_flux_update(const StepArgs& a, double* out, const double* base, double c_host, int use_dt_dev,
                               long long z) {
    int i, j, k;
    zone_ijk(a.grid, z, i, j, k);
    const R gamma = arg_gamma<R>(a), gm1 = arg_gm1<R>(a);
    double acc[5] = {0, 0, 0, 0, 0};
    flux_difference<SOLVER, 0, NV, R>(a, z, i, j, k, gamma, gm1, acc);
    flux_difference<SOLVER, 1, NV, R>(a, z, i, j, k, gamma, gm1, acc);
    flux_difference<SOLVER, 2, NV, R>(a, z, i, j, k, gamma, gm1, acc);
    store_update<R>(a, out, base, c_host, use_dt_dev, acc, z);
}

template <int SOLVER, int NV, class R>
__global__ void __launch_bounds__(128) k_flux_update(StepArgs a, double* out, const double* base, double c_host,
                                                     int use_dt_dev) {
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (z < a.grid.n) zone_flux_update<SOLVER, NV, R>(a, out, base, c_host, use_dt_dev, z);
}

// ------------------------------------------------------------------ FP32 bulk: Eq. 6 without FP64 arithmetic per face
// GB300 runs FP64 at 1/64 of the FP32 rate, so converting and differencing the twelve face fluxes of a
// zone in FP64 (about 70 FP64 instructions) bounded the FP32-bulk update.  Here the flux differences
// and their scaling by c_d = dt / dx_d are carried exactly in pairs of FP32 numbers (error-free
// transformations: Knuth's two-sum for Fm - Fp, the FMA two-product for s * c_d), so that the zone's
// increment sum_d c_d (Fm - Fp) reaches FP64 as hi + lo with a relative error near 2^-47, and only the
// accumulation U + hi + lo (and the source term) is FP64: 4 FP64 operations per variable.  c_d is split
// once per block into its FP32 head and tail.
ADER_DEV void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// true when the FP64 value is finite (exponent field not all ones), without an FP64 instruction
ADER_DEV bool finite_bits(double x) {
#ifdef __CUDA_ARCH__
    return ((__double2hiint(x) >> 20) & 0x7ff) != 0x7ff;
#else
    return isfinite(x);
#endif
}

// out = base + hi + lo (+ dt S-bar), FP64.  An addition that cannot change its FP64 sum is skipped when
// no lane of the warp needs it, so the result equals the plain sum bit for bit: hi = 0 (a zone whose
// faces all carry the same flux), and lo below half a unit in the last place of base + hi (checked on
// the exponents: |lo| < 2^(e_lo - 126) <= 2^(e_t - 1077) = ulp(t) / 2 when e_lo + 951 <= e_t).
__device__ __forceinline__ void store_pair_update(const StepArgs& a, double* out, const double* base, const float* hi,
                                                  const float* lo, long long z) {
    const long long N = a.grid.n;
    const float* Sb = (const float*)a.Sb;
    const unsigned lanes = __activemask();         // the lanes of this zone's warp still running
    bool bad = false;
    // every load before the first store (out may be base: in place)
    double b[5];
    float sb[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        b[v] = base ? base[v * N + z] : 0.0;
        sb[v] = Sb ? Sb[v * N + z] : 0.0f;
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        double val = b[v];
        if (__any_sync(lanes, hi[v] != 0.0f)) val += f64_of_f32(hi[v]);
        const unsigned e_lo = (__float_as_uint(lo[v]) >> 23) & 0xffu;
        const unsigned e_t = ((unsigned)__double2hiint(val) >> 20) & 0x7ffu;
        if (__any_sync(lanes, lo[v] != 0.0f && e_lo + 951u > e_t)) val += f64_of_f32(lo[v]);
        if (Sb) val += f64_of_f32(sb[v]);
        bad |= !finite_bits(val);
        out[v * N + z] = val;
    }
    if (bad && !a.defer_nonfinite) raise_flag(a.flag, FLAG_NONFINITE);
}

template <int SOLVER, int D, int NV>
ADER_DEV void flux_difference_pair(const StepArgs& a, long long z, int i, int j, int k, float gamma, float gm1,
                                   float chi, float clo, float* hi, float* lo) {
    const long long zm = nbr_along(a.grid, z, i, j, k, D, -1);
    const Vec<NV, float> Fp = upper_face_flux<SOLVER, D, NV, float>(a, z, i, j, k, gamma, gm1);
    const Vec<NV, float> Fm = riemann<SOLVER, D>(load_side<NV, float>(a, 2 * D, zm),
                                                 load_side<NV, float>(a, 2 * D + 1, z), gamma, gm1);
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        float s, e;
        two_sum(Fm[v], -Fp[v], s, e);                   // Fm - Fp = s + e exactly
        const float p = s * chi;
        const float pe = fmaf(s, chi, -p);              // s chi = p + pe exactly
        const float t = pe + fmaf(s, clo, e * chi);     // the small terms of (s + e)(chi + clo)
        float h, he;
        two_sum(hi[v], p, h, he);
        hi[v] = h;
        lo[v] += he + t;
    }
}

template <int SOLVER, int NV>
__global__ void __launch_bounds__(128) k_flux_update_pair(StepArgs a, double* out, const double* base, double c_host,
                                                          int use_dt_dev) {
    __shared__ float c_hi[3], c_lo[3];
    if (threadIdx.x < 3) {
        const double c = use_dt_dev ? c_host * (*a.dt_dev) : c_host;
        const double cd = c * a.idx[threadIdx.x];
        const float h = (float)cd;
        c_hi[threadIdx.x] = h;
        c_lo[threadIdx.x] = (float)(cd - (double)h);
    }
    __syncthreads();
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= a.grid.n) return;
    int i, j, k;
    zone_ijk(a.grid, z, i, j, k);
    const float gamma = a.gamma_f, gm1 = a.gm1_f;
    float hi[5] = {0, 0, 0, 0, 0}, lo[5] = {0, 0, 0, 0, 0};
    flux_difference_pair<SOLVER, 0, NV>(a, z, i, j, k, gamma, gm1, c_hi[0], c_lo[0], hi, lo);
    flux_difference_pair<SOLVER, 1, NV>(a, z, i, j, k, gamma, gm1, c_hi[1], c_lo[1], hi, lo);
    flux_difference_pair<SOLVER, 2, NV>(a, z, i, j, k, gamma, gm1, c_hi[2], c_lo[2], hi, lo);
    store_pair_update(a, out, base, hi, lo, z);
}

// The same update for one zone whose block may not share its problem (the batched kernels): c_d's FP32
// head and tail taken per zone, the split by integer conversions (one FP64 product and one difference
// per direction).
template <int SOLVER, int NV>
__device__ __forceinline__ void zone_flux_update_pair(const StepArgs& a, double* out, const double* base,
                                                      double c_host, int use_dt_dev, long long z) {
    int i, j, k;
    zone_ijk(a.grid, z, i, j, k);
    const double c = use_dt_dev ? c_host * (*a.dt_dev) : c_host;
    float chi[3], clo[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double cd = c * a.idx[d];
        chi[d] = f32_of_f64(cd);
        clo[d] = f32_of_f64(cd - f64_of_f32(chi[d]));
    }
    const float gamma = a.gamma_f, gm1 = a.gm1_f;
    float hi[5] = {0, 0, 0, 0, 0}, lo[5] = {0, 0, 0, 0, 0};
    flux_difference_pair<SOLVER, 0, NV>(a, z, i, j, k, gamma, gm1, chi[0], clo[0], hi, lo);
    flux_difference_pair<SOLVER, 1, NV>(a, z, i, j, k, gamma, gm1, chi[1], clo[1], hi, lo);
    flux_difference_pair<SOLVER, 2, NV>(a, z, i, j, k, gamma, gm1, chi[2], clo[2], hi, lo);
    store_pair_update(a, out, base, hi, lo, z);
}

template <int SOLVER, int NV, class R>
ADER_DEV void zone_face_fluxes(const StepArgs& a, long long z) {
    int i, j, k;
    zone_ijk(a.grid, z, i, j, k);
    const R gamma = arg_gamma<R>(a), gm1 = arg_gm1<R>(a);
    R* F = (R*)a.S1;
    const long long N = a.grid.n;
    const Vec<NV, R> f0 = upper_face_flux<SOLVER, 0, NV, R>(a, z, i, j, k, gamma, gm1);
#pragma unroll
    for (int v = 0; v < 5; ++v) F[(0 * 5 + v) * N + z] = f0[v];
    const Vec<NV, R> f1 = upper_face_flux<SOLVER, 1, NV, R>(a, z, i, j, k, gamma, gm1);
#pragma unroll
    for (int v = 0; v < 5; ++v) F[(1 * 5 + v) * N + z] = f1[v];
    const Vec<NV, R> f2 = upper_face_flux<SOLVER, 2, NV, R>(a, z, i, j, k, gamma, gm1);
#pragma unroll
    for (int v = 0; v < 5; ++v) F[(2 * 5 + v) * N + z] = f2[v];
}

template <int SOLVER, int NV, class R>
__global__ void __launch_bounds__(128) k_face_fluxes(StepArgs a) {
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (z < a.grid.n) zone_face_fluxes<SOLVER, NV, R>(a, z);
}

template <class R>
ADER_DEV void zone_flux_update_stored(const StepArgs& a, double* out, const double* base, double c_host,
                                      int use_dt_dev, long long z) {
    int i, j, k;
    zone_ijk(a.grid, z, i, j, k);
    const R* F = (const R*)a.S1;
    const long long N = a.grid.n;
    double acc[5] = {0, 0, 0, 0, 0};
#pragma unroll
    for (int D = 0; D < 3; ++D) {
        const long long zm = nbr_along(a.grid, z, i, j, k, D, -1);
        const double inv = a.idx[D];
#pragma unroll
        for (int v = 0; v < 5; ++v)
            acc[v] -= ((double)F[(D * 5 + v) * N + z] - (double)F[(D * 5 + v) * N + zm]) * inv;
    }
    store_update<R>(a, out, base, c_host, use_dt_dev, acc, z);
}

template <class R>
__global__ void __launch_bounds__(128) k_flux_update_stored(StepArgs a, double* out, const double* base,
                                                            double c_host, int use_dt_dev) {
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (z < a.grid.n) zone_flux_update_stored<R>(a, out, base, c_host, use_dt_dev, z);
}

// ------------------------------------------------------------------ Euler: predictor and face solves per tile
// A block owns a PT_X x PT_Y tile of (x, y) columns and marches through a chunk of z planes, one zone per
// thread and plane.  Each zone's predictor writes its six face sides (barycentre state, <u>, <F>; 15
// values each) to shared memory; after a barrier every face inside the tile is solved once, by the zone
// above it, with the side of the zone below it read from shared memory (x, y) or kept from the previous
// plane (z), and the flux is stored at the lower zone, as k_face_fluxes does: F[(D*5 + v)*N + zone] is the
// flux through the upper face of zone in direction D, in the WENO scratch S1 (each zone's modes were read
// before any flux lands on its slots).  Only the sides of the tile's and chunk's boundary zones go to
// S3, and k_tile_faces solves those faces afterwards.  The face data of the interior never reaches HBM,
// and no zone is predicted twice.
#ifndef ADER_PT_X
#define ADER_PT_X 32
#endif
#ifndef ADER_PT_Y
#define ADER_PT_Y 4
#endif
constexpr int PT_X = ADER_PT_X, PT_Y = ADER_PT_Y, PT_THREADS = PT_X * PT_Y;
constexpr int PT_NQ = 15;                     // values per Euler face side
constexpr int PT_SLOTS = 7;                   // x+, x-, y+, y-, z+ (even planes), z-, z+ (odd planes)

template <class R>
ADER_DEV R* pt_slot(R* sh, int slot, int tid) { return sh + slot * PT_NQ * PT_THREADS + tid; }

// one side into a slot: u_b (replaced by the zone mean for the wave speeds when not physical, as
// write_side does), <u>, <F>
template <class R>
ADER_DEV void pt_side(R* dst, const Vec<5, R>& mean, Vec<5, R> ub, const Vec<5, R>& avg, const Vec<5, R>& Fa, R gm1) {
    const Prim<5, R> q = primitives(ub, gm1);
    if (!(ub[0] > R(0)) || !(q.p > R(0))) ub = mean;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        dst[v * PT_THREADS] = ub[v];
        dst[(5 + v) * PT_THREADS] = avg[v];
        dst[(10 + v) * PT_THREADS] = Fa[v];
    }
}

template <int ORDER, int D, class R>
ADER_DEV void pt_sides(R* sh, int tid, int slot_plus, int slot_minus, const Vec<5, R>* m, R gm1) {
    constexpr int L = ModeCount<ORDER>::L;
    if constexpr (ZoneOps<ORDER>::HAS_FACE_PAIR) {
        Vec<5, R> p[L + 1];
        to_face_frame<ORDER, D, +1>(m, p);
        Vec<5, R> ub[2], avg[2], Fa[2];
        ZoneOps<ORDER>::template face_pair<D>(p, gm1, ub, avg, Fa);
        pt_side(pt_slot(sh, slot_plus, tid), m[1], ub[0], avg[0], Fa[0], gm1);
        pt_side(pt_slot(sh, slot_minus, tid), m[1], ub[1], avg[1], Fa[1], gm1);
    } else {
        {
            Vec<5, R> p[L + 1];
            to_face_frame<ORDER, D, +1>(m, p);
            Vec<5, R> ub, avg, Fa;
            ZoneOps<ORDER>::template face<D>(p, gm1, ub, avg, Fa);
            pt_side(pt_slot(sh, slot_plus, tid), m[1], ub, avg, Fa, gm1);
        }
        {
            Vec<5, R> p[L + 1];
            to_face_frame<ORDER, D, -1>(m, p);
            Vec<5, R> ub, avg, Fa;
            ZoneOps<ORDER>::template face<D>(p, gm1, ub, avg, Fa);
            pt_side(pt_slot(sh, slot_minus, tid), m[1], ub, avg, Fa, gm1);
        }
    }
}

template <class R>
ADER_DEV FaceSide<5, R> pt_load(const R* sh, int slot, int tid) {
    const R* s = sh + slot * PT_NQ * PT_THREADS + tid;
    FaceSide<5, R> f;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        f.ub[v] = s[v * PT_THREADS];
        f.avg[v] = s[(5 + v) * PT_THREADS];
        f.F[v] = s[(10 + v) * PT_THREADS];
    }
    return f;
}

// Boundary sides for k_tile_faces, packed in S3 (unused otherwise on this path) so that both their
// writes and k_tile_faces's reads are coalesced.  Three arrays, each [s][q][...] with s = 0 for the
// lower side of a boundary face (the x+, y+ or z+ side of the zone below it) and s = 1 for its upper
// side, q the 15 values of a side:
//   x: [2][15][tiles_x][nz][ny]   the tile's last column (s = 0) and first column (s = 1), j fastest
//   y: [2][15][tiles_y][nz][nx]   the tile's last row and first row, i fastest
//   z: [2][15][chunks][ny][nx]    the chunk's last plane and first plane, i fastest
// Each array has at most 30 N values (tiles_x <= nx, and so on), so the three fit in S3's 90 N.
struct PtBoundary {
    long long sx, sy, sz;          // values per (s, q) slice of each array
    long long ox, oy, oz;          // offsets of the arrays in S3
};

ADER_DEV PtBoundary pt_boundary(const Grid& g, int cz) {
    const long long ntx = (g.nx + PT_X - 1) / PT_X, nty = (g.ny + PT_Y - 1) / PT_Y, ncz = (g.nz + cz - 1) / cz;
    PtBoundary b;
    b.sx = ntx * g.nz * g.ny;
    b.sy = nty * g.nz * g.nx;
    b.sz = ncz * g.ny * g.nx;
    b.ox = 0;
    b.oy = 2 * PT_NQ * b.sx;
    b.oz = b.oy + 2 * PT_NQ * b.sy;
    return b;
}

// one side from shared memory into a packed boundary array: slice stride `slice`, position `pos`
template <class R>
ADER_DEV void pt_to_boundary(R* base, long long slice, long long pos, const R* sh, int slot, int tid) {
    const R* s = sh + slot * PT_NQ * PT_THREADS + tid;
#pragma unroll
    for (int q = 0; q < PT_NQ; ++q) base[q * slice + pos] = s[q * PT_THREADS];
}

template <class R>
ADER_DEV FaceSide<5, R> pt_from_boundary(const R* base, long long slice, long long pos) {
    FaceSide<5, R> f;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        f.ub[v] = base[v * slice + pos];
        f.avg[v] = base[(5 + v) * slice + pos];
        f.F[v] = base[(10 + v) * slice + pos];
    }
    return f;
}

template <int D, class R>
ADER_DEV void pt_store_flux(const StepArgs& a, long long zl, const Vec<5, R>& f) {
    R* F = (R*)a.S1;
#pragma unroll
    for (int v = 0; v < 5; ++v) F[(D * 5 + v) * a.grid.n + zl] = f[v];
}

// grid: (tiles_x * tiles_y, ceil(nz / cz)); dynamic shared memory PT_SLOTS * PT_NQ * PT_THREADS values of R
template <int ORDER, int FORM, int SOLVER, class R, bool SRC>
__global__ void __launch_bounds__(PT_THREADS, sizeof(R) == 4 ? 3 : 1)
    k_pf_tile(StepArgs a, const double* __restrict__ U, int cz) {

    extern __shared__ __align__(16) unsigned char pt_raw[];
    R* sh = reinterpret_cast<R*>(pt_raw);
    const Grid& g = a.grid;
    const int tid = threadIdx.x, tx = tid % PT_X, ty = tid / PT_X;
    const int tiles_x = (g.nx + PT_X - 1) / PT_X;
    const int i = (int)(blockIdx.x % tiles_x) * PT_X + tx, j = (int)(blockIdx.x / tiles_x) * PT_Y + ty;
    const int k0 = (int)blockIdx.y * cz, k1 = min(k0 + cz, g.nz);
    const bool valid = i < g.nx && j < g.ny;
    const bool last_x = tx == PT_X - 1 || i == g.nx - 1, last_y = ty == PT_Y - 1 || j == g.ny - 1;
    const R gamma = arg_gamma<R>(a), gm1 = arg_gm1<R>(a);
    const long long nxy = (long long)g.nx * g.ny;
    const R dt = bulk_arg<R>(a.dt_dev ? *a.dt_dev : a.dt);     // once per thread, for every plane
    const PtBoundary bd = pt_boundary(g, cz);
    R* S3 = (R*)a.S3;
    R* bx = S3 + bd.ox;
    R* by = S3 + bd.oy;
    R* bz = S3 + bd.oz;
    const long long tile_x = blockIdx.x % tiles_x, tile_y = blockIdx.x / tiles_x, chunk = blockIdx.y;
    for (int k = k0; k < k1; ++k) {
        const long long z = (long long)k * nxy + (long long)j * g.nx + i;
        const int zp_slot = (k & 1) ? 6 : 4;          // this plane's z+ sides; the previous plane's in the other
        if (valid) {
            Vec<5, R> m[ModeCount<ORDER>::L + 1];
            zone_predict<ORDER, FORM, 5, R, SRC>(a, U, z, m, dt);
            pt_sides<ORDER, 0>(sh, tid, 0, 1, m, gm1);
            pt_sides<ORDER, 1>(sh, tid, 2, 3, m, gm1);
            pt_sides<ORDER, 2>(sh, tid, zp_slot, 5, m, gm1);
        }
        __syncthreads();
        if (valid) {
            const long long px = (tile_x * g.nz + k) * g.ny + j, py = (tile_y * g.nz + k) * g.nx + i,
                            pz = (chunk * g.ny + j) * g.nx + i;
            if (tx > 0)                                // face i - 1/2: x+ side of the zone on the left
                pt_store_flux<0>(a, z - 1, riemann<SOLVER, 0>(pt_load(sh, 0, tid - 1), pt_load(sh, 1, tid), gamma, gm1));
            else
                pt_to_boundary(bx + PT_NQ * bd.sx, bd.sx, px, sh, 1, tid);
            if (last_x) pt_to_boundary(bx, bd.sx, px, sh, 0, tid);
            if (ty > 0)
                pt_store_flux<1>(a, z - g.nx,
                                 riemann<SOLVER, 1>(pt_load(sh, 2, tid - PT_X), pt_load(sh, 3, tid), gamma, gm1));
            else
                pt_to_boundary(by + PT_NQ * bd.sy, bd.sy, py, sh, 3, tid);
            if (last_y) pt_to_boundary(by, bd.sy, py, sh, 2, tid);
            if (k > k0)
                pt_store_flux<2>(a, z - nxy,
                                 riemann<SOLVER, 2>(pt_load(sh, 10 - zp_slot, tid), pt_load(sh, 5, tid), gamma, gm1));
            else
                pt_to_boundary(bz + PT_NQ * bd.sz, bd.sz, pz, sh, 5, tid);
            if (k == k1 - 1) pt_to_boundary(bz, bd.sz, pz, sh, zp_slot, tid);
        }
        __syncthreads();
    }
}

// The faces on tile and chunk boundaries, from the sides k_pf_tile packed in S3: the tile boundaries in
// x (i = multiples of PT_X, and i = 0 against nx - 1), in y (multiples of PT_Y) and the chunk boundaries
// in z (multiples of cz).  One thread per face, the packed arrays' fastest index fastest across threads.
template <int SOLVER, class R>
__global__ void __launch_bounds__(128) k_tile_faces(StepArgs a, int cz, long long nfx, long long nfy, long long nfz) {
    const Grid& g = a.grid;
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const R gamma = arg_gamma<R>(a), gm1 = arg_gm1<R>(a);
    const long long nxy = (long long)g.nx * g.ny;
    const PtBoundary bd = pt_boundary(g, cz);
    const R* S3 = (const R*)a.S3;
    if (t < nfx) {                      // x: t = (tile * nz + k) * ny + j; lower zone in the previous tile
        const int j = (int)(t % g.ny);
        const long long r = t / g.ny;
        const int k = (int)(r % g.nz), tile = (int)(r / g.nz);
        const int ntx = (g.nx + PT_X - 1) / PT_X;
        const int tl = tile == 0 ? ntx - 1 : tile - 1;
        const int il = tile == 0 ? g.nx - 1 : tile * PT_X - 1;
        const long long pl = ((long long)tl * g.nz + k) * g.ny + j;
        const R* bx = S3 + bd.ox;
        pt_store_flux<0>(a, (long long)k * nxy + (long long)j * g.nx + il,
                         riemann<SOLVER, 0>(pt_from_boundary(bx, bd.sx, pl),
                                            pt_from_boundary(bx + PT_NQ * bd.sx, bd.sx, t), gamma, gm1));
        return;
    }
    t -= nfx;
    if (t < nfy) {                      // y: t = (tile * nz + k) * nx + i
        const int i = (int)(t % g.nx);
        const long long r = t / g.nx;
        const int k = (int)(r % g.nz), tile = (int)(r / g.nz);
        const int nty = (g.ny + PT_Y - 1) / PT_Y;
        const int tl = tile == 0 ? nty - 1 : tile - 1;
        const int jl = tile == 0 ? g.ny - 1 : tile * PT_Y - 1;
        const long long pl = ((long long)tl * g.nz + k) * g.nx + i;
        const R* by = S3 + bd.oy;
        pt_store_flux<1>(a, (long long)k * nxy + (long long)jl * g.nx + i,
                         riemann<SOLVER, 1>(pt_from_boundary(by, bd.sy, pl),
                                            pt_from_boundary(by + PT_NQ * bd.sy, bd.sy, t), gamma, gm1));
        return;
    }
    t -= nfy;
    if (t < nfz) {                      // z: t = chunk * nxy + column
        const long long col = t % nxy;
        const int chunk = (int)(t / nxy);
        const int ncz = (g.nz + cz - 1) / cz;
        const int cl = chunk == 0 ? ncz - 1 : chunk - 1;
        const int kl = chunk == 0 ? g.nz - 1 : chunk * cz - 1;
        const R* bz = S3 + bd.oz;
        pt_store_flux<2>(a, (long long)kl * nxy + col,
                         riemann<SOLVER, 2>(pt_from_boundary(bz, bd.sz, (long long)cl * nxy + col),
                                            pt_from_boundary(bz + PT_NQ * bd.sz, bd.sz, t), gamma, gm1));
    }
}

// z planes per chunk: enough blocks for every SM to hold several, at most 16 planes
inline int pt_chunk(const Grid& g) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long tiles = (long long)((g.nx + PT_X - 1) / PT_X) * ((g.ny + PT_Y - 1) / PT_Y);
    long long cz = tiles * g.nz / ((long long)sms * 12);
    if (cz < 1) cz = 1;
    if (cz > 16) cz = 16;
    return (int)cz;
}

template <int ORDER, int FORM, class R, bool SRC>
void launch_pf_tile(const StepArgs& a, const double* U, cudaStream_t st) {
    const Grid& g = a.grid;
    const int cz = pt_chunk(g);
    const int ntx = (g.nx + PT_X - 1) / PT_X, nty = (g.ny + PT_Y - 1) / PT_Y, ncz = (g.nz + cz - 1) / cz;
    const size_t smem = (size_t)PT_SLOTS * PT_NQ * PT_THREADS * sizeof(R);
    const dim3 grid((unsigned)(ntx * nty), (unsigned)ncz);
    const long long nfx = (long long)ntx * g.ny * g.nz, nfy = (long long)nty * g.nx * g.nz,
                    nfz = (long long)ncz * g.nx * g.ny;
    const long long nf = nfx + nfy + nfz;
    const unsigned fblocks = (unsigned)((nf + 127) / 128);
    if (a.solver == SOLVER_HLL) {
        auto kern = k_pf_tile<ORDER, FORM, SOLVER_HLL, R, SRC>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        kern<<<grid, PT_THREADS, smem, st>>>(a, U, cz);
        k_tile_faces<SOLVER_HLL, R><<<fblocks, 128, 0, st>>>(a, cz, nfx, nfy, nfz);
    } else {
        auto kern = k_pf_tile<ORDER, FORM, SOLVER_LINEARIZED, R, SRC>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        kern<<<grid, PT_THREADS, smem, st>>>(a, U, cz);
        k_tile_faces<SOLVER_LINEARIZED, R><<<fblocks, 128, 0, st>>>(a, cz, nfx, nfy, nfz);
    }
}

// FP32 bulk, Eq. 6 from the stored face fluxes (tiled path): the differences in FP32 pairs as in
// k_flux_update_pair, the accumulation in FP64
template <class R>
__global__ void __launch_bounds__(128) k_flux_update_stored_pair(StepArgs a, double* out, const double* base,
                                                                 double c_host, int use_dt_dev) {
    static_assert(sizeof(R) == 4, "FP32 bulk only");
    __shared__ float c_hi[3], c_lo[3];
    if (threadIdx.x < 3) {
        const double c = use_dt_dev ? c_host * (*a.dt_dev) : c_host;
        const double cd = c * a.idx[threadIdx.x];
        const float h = (float)cd;
        c_hi[threadIdx.x] = h;
        c_lo[threadIdx.x] = (float)(cd - (double)h);
    }
    __syncthreads();
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= a.grid.n) return;
    int i, j, k;
    zone_ijk(a.grid, z, i, j, k);
    const float* F = (const float*)a.S1;
    const long long N = a.grid.n;
    float hi[5] = {0, 0, 0, 0, 0}, lo[5] = {0, 0, 0, 0, 0};
#pragma unroll
    for (int D = 0; D < 3; ++D) {
        const long long zm = nbr_along(a.grid, z, i, j, k, D, -1);
        const float chi = c_hi[D], clo = c_lo[D];
#pragma unroll
        for (int v = 0; v < 5; ++v) {
            float s, e;
            two_sum(F[(D * 5 + v) * N + zm], -F[(D * 5 + v) * N + z], s, e);
            const float p = s * chi;
            const float pe = fmaf(s, chi, -p);
            const float t = pe + fmaf(s, clo, e * chi);
            float h, he;
            two_sum(hi[v], p, h, he);
            hi[v] = h;
            lo[v] += he + t;
        }
    }
    store_pair_update(a, out, base, hi, lo, z);
}

// ------------------------------------------------------------------ MHD: edge EMFs (Sec. II.3, Eq. 7)
// HLL flux of the face of direction D between zones zl (lower) and zr,
// evaluated with its edge slot e (0: t1+, 1: t1-, 2: t2+, 3: t2-): the face's
// own frozen wave speeds (from its barycentre states) applied to the edge
// averages of its two sides.
// A face's Riemann problem is transonic when a fast wave speed changes sign between its two states.
template <class R>
ADER_DEV bool transonic(R vl, R cl, R vr, R cr) {
    return (vl - cl) * (vr - cr) < R(0) || (vl + cl) * (vr + cr) < R(0);
}

template <int D, class R>
ADER_DEV R edge_hll(const StepArgs& a, long long zl, long long zr, int e, R gamma, R gm1) {
    constexpr int NQ = side_values(8);
    const R* S3 = (const R*)a.S3;
    const long long N = a.grid.n;
    const int sl = 2 * D, sr = 2 * D + 1;
    Vec<8, R> ubl, ubr;
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        ubl[v] = S3[(sl * NQ + v) * N + zl];
        ubr[v] = S3[(sr * NQ + v) * N + zr];
    }
    const Prim<8, R> pl = primitives(ubl, gm1), pr = primitives(ubr, gm1);
    const R vl = D == 0 ? pl.vx : (D == 1 ? pl.vy : pl.vz);
    const R vr = D == 0 ? pr.vx : (D == 1 ? pr.vy : pr.vz);
    const R cl = fast_speed<D>(ubl, pl, gamma), cr = fast_speed<D>(ubr, pr, gamma);
    const R lamL = fmin(fmin(vl - cl, vr - cr), R(0));
    const R lamR = fmax(fmax(vl + cl, vr + cr), R(0));
    const R uL = S3[(sl * NQ + 24 + 2 * e) * N + zl], FL = S3[(sl * NQ + 25 + 2 * e) * N + zl];
    const R uR = S3[(sr * NQ + 24 + 2 * e) * N + zr], FR = S3[(sr * NQ + 25 + 2 * e) * N + zr];
    // optional: twice the third (dissipative) term of Eq. 17 where a fast speed changes sign (Sec. V)
    const R w = (a.emf_transonic && transonic(vl, cl, vr, cr)) ? R(2) : R(1);
    return (lamR * FL - lamL * FR + (w * lamR) * lamL * (uR - uL)) / (lamR - lamL);
}

// The same flux with the linearized solver: |A| at the mean of the face's two
// barycentre states applied to the jump of the full edge-averaged states.
template <int D, class R>
ADER_DEV R edge_linearized(const StepArgs& a, long long zl, long long zr, int e, R gamma, R gm1) {
    constexpr int NQ = side_values(8);
    constexpr int T1 = D == 0 ? 1 : 0, T2 = D == 2 ? 1 : 2;
    const R* S3 = (const R*)a.S3;
    const R* X = S3 + (long long)6 * NQ * a.grid.n;
    const long long N = a.grid.n;
    const int sl = 2 * D, sr = 2 * D + 1;
    Vec<8, R> ubl, ubr, dU;
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        ubl[v] = S3[(sl * NQ + v) * N + zl];
        ubr[v] = S3[(sr * NQ + v) * N + zr];
        dU[v] = X[(sr * EDGE_STATE_VALUES + e * 8 + v) * N + zr] - X[(sl * EDGE_STATE_VALUES + e * 8 + v) * N + zl];
    }
    const MeanState<R> m = mhd_mean_state(ubl, ubr, gm1);
    const Vec<8, R> diss = mhd_abs_jacobian_apply<D, R>(m.rho, m.v, m.p, m.B, gamma, gm1, dU);
    const int c = 5 + (e < 2 ? T1 : T2);
    const R FL = S3[(sl * NQ + 25 + 2 * e) * N + zl], FR = S3[(sr * NQ + 25 + 2 * e) * N + zr];
    R w = R(1);
    if (a.emf_transonic) {           // optional doubled dissipation at transonic faces (Sec. V)
        const Prim<8, R> pl = primitives(ubl, gm1), pr = primitives(ubr, gm1);
        const R vl = D == 0 ? pl.vx : (D == 1 ? pl.vy : pl.vz);
        const R vr = D == 0 ? pr.vx : (D == 1 ? pr.vy : pr.vz);
        if (transonic(vl, fast_speed<D>(ubl, pl, gamma), vr, fast_speed<D>(ubr, pr, gamma))) w = R(2);
    }
    return R(0.5) * (FL + FR) - (R(0.5) * w) * diss[c];
}

template <int D, class R>
ADER_DEV R edge_flux(const StepArgs& a, long long zl, long long zr, int e, R gamma, R gm1) {
    return a.solver == SOLVER_LINEARIZED ? edge_linearized<D, R>(a, zl, zr, e, gamma, gm1)
                                         : edge_hll<D, R>(a, zl, zr, e, gamma, gm1);
}

// EMFs at the three upper edges of zone (i, j, k): Ez on (i+1/2, j+1/2),
// Ey on (i+1/2, k+1/2), Ex on (j+1/2, k+1/2); each the mean of the four
// adjacent faces' edge fluxes with Eq. 7's signs (Ez = -F7 = G6,
// Ey = F8 = -H6, Ex = -G8 = H7).
template <class R>
ADER_DEV void zone_emf(const StepArgs& a, long long z) {
    const Grid& g = a.grid;
    int i, j, k;
    zone_ijk(g, z, i, j, k);
    const R gamma = arg_gamma<R>(a), gm1 = arg_gm1<R>(a);
    const long long zx = nbr(g, i, j, k, 1, 0, 0), zy = nbr(g, i, j, k, 0, 1, 0), zz = nbr(g, i, j, k, 0, 0, 1);
    const long long zxy = nbr(g, i, j, k, 1, 1, 0), zxz = nbr(g, i, j, k, 1, 0, 1), zyz = nbr(g, i, j, k, 0, 1, 1);
    // x-faces: t1 = y (slots 0, 1), t2 = z (2, 3); y-faces: t1 = x, t2 = z; z-faces: t1 = x, t2 = y
    const R Ez = R(0.25) * (-edge_flux<0, R>(a, z, zx, 0, gamma, gm1) - edge_flux<0, R>(a, zy, zxy, 1, gamma, gm1) +
                            edge_flux<1, R>(a, z, zy, 0, gamma, gm1) + edge_flux<1, R>(a, zx, zxy, 1, gamma, gm1));
    const R Ey = R(0.25) * (edge_flux<0, R>(a, z, zx, 2, gamma, gm1) + edge_flux<0, R>(a, zz, zxz, 3, gamma, gm1) -
                            edge_flux<2, R>(a, z, zz, 0, gamma, gm1) - edge_flux<2, R>(a, zx, zxz, 1, gamma, gm1));
    const R Ex = R(0.25) * (-edge_flux<1, R>(a, z, zy, 2, gamma, gm1) - edge_flux<1, R>(a, zz, zyz, 3, gamma, gm1) +
                            edge_flux<2, R>(a, z, zz, 2, gamma, gm1) + edge_flux<2, R>(a, zy, zyz, 3, gamma, gm1));
    R* E = (R*)a.E;
    E[z] = Ex;
    E[g.n + z] = Ey;
    E[2 * g.n + z] = Ez;
}

template <class R>
__global__ void __launch_bounds__(128) k_emf(StepArgs a) {
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (z < a.grid.n) zone_emf<R>(a, z);
}

// Eq. 8 on the three faces i-1/2, j-1/2, k-1/2 of zone (i, j, k): each face
// is written by exactly one zone, so the update is in place.
template <class R>
ADER_DEV void zone_ct(const StepArgs& a, double* Bf, double c_host, int use_dt_dev, long long z) {
    const Grid& g = a.grid;
    int i, j, k;
    zone_ijk(g, z, i, j, k);
    const R* E = (const R*)a.E;
    const long long N = g.n;
    // FP32 edge fields widen to FP64 exactly on the integer pipe (f64_of_f32), not by conversions on the
    // FP64 units
    auto wide = [](R e) -> double {
        if constexpr (sizeof(R) == 4) return f64_of_f32(e); else return e;
    };
    auto Ex = [&](int di, int dj, int dk) { return wide(E[nbr(g, i, j, k, di, dj, dk)]); };
    auto Ey = [&](int di, int dj, int dk) { return wide(E[N + nbr(g, i, j, k, di, dj, dk)]); };
    auto Ez = [&](int di, int dj, int dk) { return wide(E[2 * N + nbr(g, i, j, k, di, dj, dk)]); };
    const double dt = use_dt_dev ? c_host * (*a.dt_dev) : c_host;
    const double idx = a.idx[0], idy = a.idx[1], idz = a.idx[2];
    // the edges of face i-1/2 are stored one zone lower in x (likewise for y, z)
    Bf[z] -= dt * ((Ez(-1, 0, 0) - Ez(-1, -1, 0)) * idy - (Ey(-1, 0, 0) - Ey(-1, 0, -1)) * idz);
    Bf[N + z] -= dt * ((Ex(0, -1, 0) - Ex(0, -1, -1)) * idz - (Ez(0, -1, 0) - Ez(-1, -1, 0)) * idx);
    Bf[2 * N + z] -= dt * ((Ey(0, 0, -1) - Ey(-1, 0, -1)) * idx - (Ex(0, 0, -1) - Ex(0, -1, -1)) * idy);
}

template <class R>
__global__ void __launch_bounds__(128) k_ct(StepArgs a, double* Bf, double c_host, int use_dt_dev) {
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (z < a.grid.n) zone_ct<R>(a, Bf, c_host, use_dt_dev, z);
}

// One variant of the predictor + face kernel, launched over the grid.  Each variant can be compiled in a
// translation unit of its own (the fourth-order ones are, see step_inst.cuh), which keeps the parallel
// build's longest compile short.
template <int ORDER, int FORM, int NV, class R, bool SRC>
void launch_pf_variant(const StepArgs& a, const double* U, cudaStream_t st) {
    if constexpr (NV == 5 && ORDER <= 3) {
        if (a.tiled) {
            launch_pf_tile<ORDER, FORM, R, SRC>(a, U, st);
            return;
        }
    }
    const int T = 128;
    const unsigned blocks = (unsigned)((a.grid.n + T - 1) / T);
    k_predict_faces<ORDER, FORM, NV, R, SRC><<<blocks, T, 0, st>>>(a, U);
}

template <int ORDER, int NV, class R>
int launch_predict_faces_nv(const StepArgs& a, const double* U, cudaStream_t st) {
    if constexpr (ZoneOps<ORDER>::HAS_SOURCE) {
        if (a.src_kind != SOURCE_NONE && a.Sb && a.n_iter > 0) {
            if (a.form == FORM_NODAL) {
                launch_pf_variant<ORDER, FORM_NODAL, NV, R, true>(a, U, st);
                return (NV == 5 && ORDER <= 3 && a.tiled) ? 2 : 1;
            }
            if constexpr (ZoneOps<ORDER>::HAS_SOURCE_MODAL) {
                launch_pf_variant<ORDER, FORM_MODAL, NV, R, true>(a, U, st);
                return (NV == 5 && ORDER <= 3 && a.tiled) ? 2 : 1;
            }
        }
    }
    if (a.form == FORM_MODAL)
        launch_pf_variant<ORDER, FORM_MODAL, NV, R, false>(a, U, st);
    else
        launch_pf_variant<ORDER, FORM_NODAL, NV, R, false>(a, U, st);
    return (NV == 5 && ORDER <= 3 && a.tiled) ? 2 : 1;
}

}  // namespace ader
