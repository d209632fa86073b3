// FP64 reductions: the CFL time step (warp shuffles, one launch with a
// last-block finish) and the conservation totals (deterministic two passes);
// plus the flux-update launcher and the state linear combination of SSP-RK.
#include "kernels.cuh"
#include "step_kernels.cuh"

namespace ader {

// dt = cfl / max over zones of sum_d (|v_d| + a) / dx_d (reading of the CFL rule).
// scratch[0]: running maximum as the bit pattern of a non-negative double
// (ordered like an unsigned integer); scratch[1]: blocks finished.  The last
// block to finish writes dt and resets both words for the next call.
// For MHD (Bf non-null) c_d is the fast speed of the zone state whose field is the mean of the
// two face values (Sec. III, opening).
// S is the precision of the per-zone signal speed: FP64, or FP32 for FP32-bulk
// contexts (there FP64's division and square root would dominate the kernel);
// the maximum, its reduction and dt are FP64 in both.
// The state in the precision S of the signal speeds; FP32 rounds with integer operations (f32_of_f64).
template <class S>
__device__ __forceinline__ S speed_operand(double x) {
    if constexpr (sizeof(S) == 4)
        return f32_of_f64(x);
    else
        return x;
}

template <class S>
__global__ void __launch_bounds__(256) k_max_dt(Grid g, const double* __restrict__ U, const double* __restrict__ Bf,
                                                double gamma, double idx, double idy, double idz, double cfl,
                                                double* dt_out, unsigned long long* scratch, unsigned* flag) {
    S sm = S(0);                       // the largest signal-speed sum of this thread, in S (FP64 below)
    bool bad = false;
    const long long N = g.n;
    const S gm = S(gamma), ix = S(idx), iy = S(idy), iz = S(idz);
    const long long stride = (long long)gridDim.x * blockDim.x;
    // four zones per pass, their twenty loads issued before any arithmetic (more bytes in flight)
    for (long long z0 = (long long)blockIdx.x * blockDim.x + threadIdx.x; z0 < N; z0 += 4 * stride) {
    double ld[4][5];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const long long zz = z0 + u * stride;
#pragma unroll
        for (int c = 0; c < 5; ++c) ld[u][c] = zz < N ? U[c * N + zz] : 1.0;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const long long z = z0 + u * stride;
        if (z >= N) break;
        const S rho = speed_operand<S>(ld[u][0]), mx = speed_operand<S>(ld[u][1]), my = speed_operand<S>(ld[u][2]),
                mz = speed_operand<S>(ld[u][3]), E = speed_operand<S>(ld[u][4]);
        const S ir = S(1) / rho;
        const S vx = mx * ir, vy = my * ir, vz = mz * ir;
        S v;
        if (Bf) {
            int i, j, k;
            zone_ijk(g, z, i, j, k);
            Vec<8, S> u;
            u[0] = rho; u[1] = mx; u[2] = my; u[3] = mz; u[4] = E;
            u[5] = S(0.5 * (Bf[z] + Bf[nbr(g, i, j, k, 1, 0, 0)]));
            u[6] = S(0.5 * (Bf[N + z] + Bf[N + nbr(g, i, j, k, 0, 1, 0)]));
            u[7] = S(0.5 * (Bf[2 * N + z] + Bf[2 * N + nbr(g, i, j, k, 0, 0, 1)]));
            const Prim<8, S> q = primitives(u, gm - S(1));
            if (!(rho > S(0)) || !(q.p > S(0))) {
                bad = true;
                continue;
            }
            v = (fabs(vx) + fast_speed<0>(u, q, gm)) * ix + (fabs(vy) + fast_speed<1>(u, q, gm)) * iy +
                (fabs(vz) + fast_speed<2>(u, q, gm)) * iz;
        } else {
            const S p = (gm - S(1)) * (E - S(0.5) * (mx * vx + my * vy + mz * vz));
            if (!(rho > S(0)) || !(p > S(0))) {
                bad = true;
                continue;
            }
            const S a = sqrt(gm * p * ir);
            v = (fabs(vx) + a) * ix + (fabs(vy) + a) * iy + (fabs(vz) + a) * iz;
        }
        sm = fmax(sm, v);
    }
    }
    double s = (double)sm;
    if (bad) raise_flag(flag, FLAG_UNPHYSICAL);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
    __shared__ double warp_max[8];
    __shared__ bool last;
    if ((threadIdx.x & 31) == 0) warp_max[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b = fmax(b, warp_max[w]);
        atomicMax(&scratch[0], (unsigned long long)__double_as_longlong(b));
        __threadfence();
        const unsigned long long done = atomicAdd(&scratch[1], 1ull);
        last = (done == gridDim.x - 1);
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        const double mx = __longlong_as_double((long long)atomicAdd(&scratch[0], 0ull));
        *dt_out = mx > 0.0 ? cfl / mx : 0.0;
        scratch[0] = 0ull;
        scratch[1] = 0ull;
    }
}

int launch_max_dt(const Grid& g, const double* U, const double* Bf, double gamma, const double dx[3], double cfl,
                  double* dt_dev, unsigned long long* scratch, unsigned* flag, bool fp32, cudaStream_t st) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long want = (g.n + 1023) / 1024;                 // four zones per thread and pass
    const long long cap = (long long)sms * 8;
    const unsigned blocks = (unsigned)(want < cap ? (want > 0 ? want : 1) : cap);
    if (fp32)
        k_max_dt<float><<<blocks, 256, 0, st>>>(g, U, Bf, gamma, 1.0 / dx[0], 1.0 / dx[1], 1.0 / dx[2], cfl, dt_dev,
                                                scratch, flag);
    else
        k_max_dt<double><<<blocks, 256, 0, st>>>(g, U, Bf, gamma, 1.0 / dx[0], 1.0 / dx[1], 1.0 / dx[2], cfl, dt_dev,
                                                 scratch, flag);
    return 1;
}

// ---------------------------------------------------------------- totals
__global__ void __launch_bounds__(256) k_totals_partial(Grid g, const double* __restrict__ U, double* partial) {
    double s[5] = {0, 0, 0, 0, 0};
    const long long N = g.n;
    for (long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x; z < N; z += (long long)gridDim.x * blockDim.x)
#pragma unroll
        for (int v = 0; v < 5; ++v) s[v] += U[v * N + z];
    __shared__ double sh[5][256];
#pragma unroll
    for (int v = 0; v < 5; ++v) sh[v][threadIdx.x] = s[v];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
#pragma unroll
            for (int v = 0; v < 5; ++v) sh[v][threadIdx.x] += sh[v][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 5) partial[blockIdx.x * 5 + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void k_totals_final(const double* partial, int nblocks, double* out) {
    if (threadIdx.x < 5) {
        double s = 0.0;
        for (int b = 0; b < nblocks; ++b) s += partial[b * 5 + threadIdx.x];
        out[threadIdx.x] = s;
    }
}

// MHD: totals of the five zone variables and of the three face-field arrays,
// plus the largest |div B| of a zone (the discrete divergence that Eq. 8
// keeps constant) and the largest |B| on a face.  partial holds 10 values per
// block: 8 sums, then the two maxima.
__global__ void __launch_bounds__(256) k_diag_mhd_partial(Grid g, const double* __restrict__ U,
                                                          const double* __restrict__ Bf, double idx, double idy,
                                                          double idz, double* partial) {
    double s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    double dmax = 0.0, bmax = 0.0;
    const long long N = g.n;
    for (long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x; z < N; z += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int v = 0; v < 5; ++v) s[v] += U[v * N + z];
        int i, j, k;
        zone_ijk(g, z, i, j, k);
        const double bx = Bf[z], by = Bf[N + z], bz = Bf[2 * N + z];
        s[5] += bx;
        s[6] += by;
        s[7] += bz;
        const double div = (Bf[nbr(g, i, j, k, 1, 0, 0)] - bx) * idx + (Bf[N + nbr(g, i, j, k, 0, 1, 0)] - by) * idy +
                           (Bf[2 * N + nbr(g, i, j, k, 0, 0, 1)] - bz) * idz;
        dmax = fmax(dmax, fabs(div));
        bmax = fmax(bmax, fmax(fabs(bx), fmax(fabs(by), fabs(bz))));
    }
    __shared__ double sh[10][256];
#pragma unroll
    for (int v = 0; v < 8; ++v) sh[v][threadIdx.x] = s[v];
    sh[8][threadIdx.x] = dmax;
    sh[9][threadIdx.x] = bmax;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
#pragma unroll
            for (int v = 0; v < 8; ++v) sh[v][threadIdx.x] += sh[v][threadIdx.x + w];
            sh[8][threadIdx.x] = fmax(sh[8][threadIdx.x], sh[8][threadIdx.x + w]);
            sh[9][threadIdx.x] = fmax(sh[9][threadIdx.x], sh[9][threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x < 10) partial[blockIdx.x * 10 + threadIdx.x] = sh[threadIdx.x][0];
}

// out[0..7] = totals, out[8] = max |div B| / (max |B| / min(dx, dy, dz)) (0 when B = 0)
__global__ void k_diag_mhd_final(const double* partial, int nblocks, double dxmin, double* out) {
    const int v = threadIdx.x;
    if (v < 8) {
        double s = 0.0;
        for (int b = 0; b < nblocks; ++b) s += partial[b * 10 + v];
        out[v] = s;
    } else if (v == 8) {
        double dm = 0.0, bm = 0.0;
        for (int b = 0; b < nblocks; ++b) {
            dm = fmax(dm, partial[b * 10 + 8]);
            bm = fmax(bm, partial[b * 10 + 9]);
        }
        out[8] = bm > 0.0 ? dm * dxmin / bm : 0.0;
    }
}

int launch_totals(const Grid& g, const double* U, const double* Bf, const double dx[3], double* totals_dev,
                  double* partial, int nblocks, cudaStream_t st) {
    if (Bf) {
        const double dxmin = fmin(dx[0], fmin(dx[1], dx[2]));
        k_diag_mhd_partial<<<nblocks, 256, 0, st>>>(g, U, Bf, 1.0 / dx[0], 1.0 / dx[1], 1.0 / dx[2], partial);
        k_diag_mhd_final<<<1, 32, 0, st>>>(partial, nblocks, dxmin, totals_dev);
        return 2;
    }
    k_totals_partial<<<nblocks, 256, 0, st>>>(g, U, partial);
    k_totals_final<<<1, 32, 0, st>>>(partial, nblocks, totals_dev);
    return 2;
}

// ---------------------------------------------------------------- SSP-RK combination
struct Comb {
    const double* X[6];
    double c[6];
    int n;
};

__global__ void __launch_bounds__(256) k_lincomb(double* out, Comb cb, long long count) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int t = 0; t < cb.n; ++t) s += cb.c[t] * cb.X[t][i];
        out[i] = s;
    }
}

int launch_lincomb(double* out, int n, const double* const* X, const double* c, long long count, cudaStream_t st) {
    Comb cb;
    cb.n = n;
    for (int t = 0; t < n; ++t) {
        cb.X[t] = X[t];
        cb.c[t] = c[t];
    }
    const long long blocks = (count + 255) / 256;
    k_lincomb<<<(unsigned)(blocks < 152 * 16 ? blocks : 152 * 16), 256, 0, st>>>(out, cb, count);
    return 1;
}

// ---------------------------------------------------------------- flux + update
template <class R>
int launch_flux_update(const StepArgs& a, double* out, const double* base, double c_host, bool use_dt_dev,
                       cudaStream_t st) {
    const int T = 128;
    const unsigned blocks = (unsigned)((a.grid.n + T - 1) / T);
    const int dd = use_dt_dev ? 1 : 0;
    if (!a.mhd && a.order <= 3 && a.tiled) {   // the tile kernel stored every face flux once
        if constexpr (sizeof(R) == 4)
            k_flux_update_stored_pair<R><<<blocks, T, 0, st>>>(a, out, base, c_host, dd);
        else
            k_flux_update_stored<R><<<blocks, T, 0, st>>>(a, out, base, c_host, dd);
        return 1;
    }
    if constexpr (sizeof(R) == 4) {           // fused, both faces of each direction per zone, FP32 pairs
        if (a.mhd && a.solver == SOLVER_HLL)
            k_flux_update_pair<SOLVER_HLL, 8><<<blocks, T, 0, st>>>(a, out, base, c_host, dd);
        else if (a.mhd)
            k_flux_update_pair<SOLVER_LINEARIZED, 8><<<blocks, T, 0, st>>>(a, out, base, c_host, dd);
        else if (a.solver == SOLVER_HLL)
            k_flux_update_pair<SOLVER_HLL, 5><<<blocks, T, 0, st>>>(a, out, base, c_host, dd);
        else
            k_flux_update_pair<SOLVER_LINEARIZED, 5><<<blocks, T, 0, st>>>(a, out, base, c_host, dd);
        return 1;
    } else {                                   // each face solved once, then the update
        if (a.mhd && a.solver == SOLVER_HLL)
            k_face_fluxes<SOLVER_HLL, 8, R><<<blocks, T, 0, st>>>(a);
        else if (a.mhd)
            k_face_fluxes<SOLVER_LINEARIZED, 8, R><<<blocks, T, 0, st>>>(a);
        else if (a.solver == SOLVER_HLL)
            k_face_fluxes<SOLVER_HLL, 5, R><<<blocks, T, 0, st>>>(a);
        else
            k_face_fluxes<SOLVER_LINEARIZED, 5, R><<<blocks, T, 0, st>>>(a);
        k_flux_update_stored<R><<<blocks, T, 0, st>>>(a, out, base, c_host, dd);
        return 2;
    }
}

template <class R>
int launch_emf_ct(const StepArgs& a, double* Bf, double c_host, bool use_dt_dev, cudaStream_t st) {
    const int T = 128;
    const unsigned blocks = (unsigned)((a.grid.n + T - 1) / T);
    k_emf<R><<<blocks, T, 0, st>>>(a);
    k_ct<R><<<blocks, T, 0, st>>>(a, Bf, c_host, use_dt_dev ? 1 : 0);
    return 2;
}

template int launch_flux_update<double>(const StepArgs&, double*, const double*, double, bool, cudaStream_t);
template int launch_flux_update<float>(const StepArgs&, double*, const double*, double, bool, cudaStream_t);
template int launch_emf_ct<double>(const StepArgs&, double*, double, bool, cudaStream_t);
template int launch_emf_ct<float>(const StepArgs&, double*, double, bool, cudaStream_t);

}  // namespace ader
