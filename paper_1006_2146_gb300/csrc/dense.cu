// Dense output inside a step (Sec. VII): the predictor's space-time polynomial restricted to a time.
//
// A step that keeps its modes (StepArgs::modes_out) leaves u_k, k = 1..L, of every zone:
// u(xi, eta, zeta, tau) = sum_k u_k P_a(xi) P_b(eta) P_c(zeta) tau^d (Eqs. 9, 13, 14-16).  At a fixed
// tau in [0, 1] this is a spatial polynomial with modes w_s = sum over the k with spatial part s of
// u_k tau^{d_k}; w_1 is the zone average (every P_a with a >= 1 has zero mean).  One thread per zone,
// FP64 output; the work is a handful of FMAs per value, so the kernel runs at the memory rate.
#include <utility>

#include "kernels.cuh"
#include "modes.cuh"

namespace ader {

// Mode K (> LS) of order ORDER: the index of its spatial part and its time degree, as compile-time
// constants (the mode tables are host constexpr arrays, which device code may only read in constant
// expressions).
template <int ORDER, int K>
struct TimeMode {
    static constexpr Exp4 e = mode_exp<ORDER>(K);
    static constexpr int s = find_mode<ORDER>(e.a, e.b, e.c, 0);
    static constexpr int d = e.d;
};

template <int ORDER, int NV, class R, int... J>
ADER_DEV void add_time_modes(double* w, const R* __restrict__ modes, int v, long long N, long long z,
                             const double* tp, std::integer_sequence<int, J...>) {
    constexpr int LS = ModeCount<ORDER>::LS;
    ((w[TimeMode<ORDER, LS + 1 + J>::s] +=
      (double)modes[(long long)((LS + J) * NV + v) * N + z] * tp[TimeMode<ORDER, LS + 1 + J>::d]), ...);
}

template <int ORDER, int NV, class R>
ADER_DEV void zone_dense_eval(const R* __restrict__ modes, long long N, double tau, double* __restrict__ out,
                              long long z) {
    constexpr int LS = ModeCount<ORDER>::LS, L = ModeCount<ORDER>::L;
    double tp[ORDER];           // tau^d, d < ORDER (the time degree is at most M - 1)
    tp[0] = 1.0;
#pragma unroll
    for (int d = 1; d < ORDER; ++d) tp[d] = tp[d - 1] * tau;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        double w[LS + 1];
#pragma unroll
        for (int s = 1; s <= LS; ++s) w[s] = (double)modes[(long long)((s - 1) * NV + v) * N + z];
        add_time_modes<ORDER, NV, R>(w, modes, v, N, z, tp, std::make_integer_sequence<int, L - LS>{});
#pragma unroll
        for (int s = 1; s <= LS; ++s) out[(long long)((s - 1) * NV + v) * N + z] = w[s];
    }
}

template <int ORDER, int NV, class R>
__global__ void __launch_bounds__(128) k_dense_eval(const R* __restrict__ modes, long long N, double tau,
                                                    double* __restrict__ out) {
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (z < N) zone_dense_eval<ORDER, NV, R>(modes, N, tau, out, z);
}

template <int ORDER, int NV, class R>
static void launch_one(const void* modes, long long N, double tau, double* out, cudaStream_t st) {
    const int T = 128;
    const unsigned blocks = (unsigned)((N + T - 1) / T);
    k_dense_eval<ORDER, NV, R><<<blocks, T, 0, st>>>((const R*)modes, N, tau, out);
}

template <int NV, class R>
static void launch_nv(int order, const void* modes, long long N, double tau, double* out, cudaStream_t st) {
    if (order == 2) launch_one<2, NV, R>(modes, N, tau, out, st);
    else if (order == 3) launch_one<3, NV, R>(modes, N, tau, out, st);
    else launch_one<4, NV, R>(modes, N, tau, out, st);
}

int launch_dense_eval(int order, int nv, bool fp32, const void* modes, long long N, double tau, double* out,
                      cudaStream_t st) {
    if (N <= 0) return 0;
    if (nv == 8) {
        if (fp32) launch_nv<8, float>(order, modes, N, tau, out, st);
        else launch_nv<8, double>(order, modes, N, tau, out, st);
    } else {
        if (fp32) launch_nv<5, float>(order, modes, N, tau, out, st);
        else launch_nv<5, double>(order, modes, N, tau, out, st);
    }
    return 1;
}

}  // namespace ader
