// Training and data generation of the learned predictor guess (see mlp.cuh).
//
// Data: for every zone of a state, the features and the normalised targets
// of the CONVERGED FP64 predictor started from zero (modal, third order).
// Training: mean-squared error, minibatch Adam, FP32, with the project's own
// kernels: a tiled GEMM (C = op(A) op(B) [+ C]), bias + GELU forward and
// backward, column sums for the bias gradients, and the Adam update.
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/ader.h"
#include "kernels.cuh"
#include "mlp.cuh"
#include "step_inst.cuh"
#include "weno.cuh"

namespace ader {

// ---------------------------------------------------------------- samples
template <int NV>
__global__ void __launch_bounds__(128) k_guess_samples(StepArgs a, const double* __restrict__ U, float* X, float* Y,
                                                       int* ok) {
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= a.grid.n) return;
    Vec<NV, double> m[16];
    load_modes<3>(a, U, z, m);
#pragma unroll
    for (int k = 11; k <= 15; ++k) m[k] = vzero<NV, double>();
    const double dt = a.dt;
    const double cx = dt / a.dx[0], cy = dt / a.dx[1], cz = dt / a.dx[2];
    const GuessScales<NV, double> g = guess_scales<NV, double>(m, cx, cy, cz);
    float* x = X + z * mlp_in(NV);
    float* y = Y + z * mlp_out(NV);
    const double mag = g.ok ? guess_features<NV, double>(m, g, cx, cy, cz, x) : 0.0;
    PredCtl ctl{2, a.tol, a.max_iter, 0, false};
    o3::predict_modal(m, a.gamma - 1.0, cx, cy, cz, ctl);
    const bool use = g.ok && mag > GUESS_MAG_MIN && !ctl.capped;
    if (use) guess_targets<NV, double>(m, g, mag, y);
    ok[z] = use ? 1 : 0;
}

// ---------------------------------------------------------------- GEMM
// C[M x N] = sum_k A(i, k) B(k, j) (+ C if accumulate), FP32.
// A(i, k) = A[i*lda + k] (ta = 0) or A[k*lda + i] (ta = 1); likewise B(k, j) = B[k*ldb + j] or B[j*ldb + k].
constexpr int GT = 64, GK = 16;

__global__ void __launch_bounds__(256) k_gemm(int M, int N, int K, const float* __restrict__ A, int lda, int ta,
                                              const float* __restrict__ B, int ldb, int tb, float* C, int ldc,
                                              int accumulate) {
    __shared__ float As[GK][GT + 4];
    __shared__ float Bs[GK][GT + 4];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int row0 = blockIdx.y * GT, col0 = blockIdx.x * GT;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += GK) {
        for (int e = threadIdx.x; e < GT * GK; e += 256) {
            const int r = e / GK, kk = e % GK;               // A tile: rows r, cols kk
            const int gi = row0 + r, gk = k0 + kk;
            As[kk][r] = (gi < M && gk < K) ? (ta ? A[(long long)gk * lda + gi] : A[(long long)gi * lda + gk]) : 0.f;
            const int c = e / GK, kb = e % GK;               // B tile: cols c, rows kb
            const int gj = col0 + c, gkb = k0 + kb;
            Bs[kb][c] = (gj < N && gkb < K) ? (tb ? B[(long long)gj * ldb + gkb] : B[(long long)gkb * ldb + gj]) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                a[q] = As[kk][ty * 4 + q];
                b[q] = Bs[kk][tx * 4 + q];
            }
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(a[p], b[q], acc[p][q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int i = row0 + ty * 4 + p;
        if (i >= M) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int j = col0 + tx * 4 + q;
            if (j >= N) continue;
            float* cp = C + (long long)i * ldc + j;
            *cp = accumulate ? *cp + acc[p][q] : acc[p][q];
        }
    }
}

static void gemm(int M, int N, int K, const float* A, int lda, int ta, const float* B, int ldb, int tb, float* C,
                 int ldc, int accumulate, cudaStream_t st) {
    dim3 grid((N + GT - 1) / GT, (M + GT - 1) / GT);
    k_gemm<<<grid, 256, 0, st>>>(M, N, K, A, lda, ta, B, ldb, tb, C, ldc, accumulate);
}

// Z[r][c] += b[c]; H = gelu(Z) (H may be null: linear output layer)
__global__ void k_bias_act(float* Z, float* H, const float* b, long long rows, int cols) {
    const long long n = rows * cols;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const float z = Z[e] + b[e % cols];
        Z[e] = z;
        if (H) H[e] = gelu(z);
    }
}

// dY = 2 (Yp - Y) / (rows * cols); partial loss sums per block (FP64)
__global__ void k_mse(const float* Yp, const float* Y, float* dY, long long n, float scale, double* loss_partial) {
    double s = 0.0;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const float d = Yp[e] - Y[e];
        s += (double)d * d;
        if (dY) dY[e] = 2.0f * d * scale;
    }
    __shared__ double sh[256];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss_partial[blockIdx.x] = sh[0];
}

// dZ = dH * gelu'(Z)
__global__ void k_gelu_back(const float* dH, const float* Z, float* dZ, long long n) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        dZ[e] = dH[e] * gelu_grad(Z[e]);
}

// db[c] = sum_r dZ[r][c]
__global__ void k_colsum(const float* dZ, float* db, long long rows, int cols) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    float s = 0.f;
    for (long long r = 0; r < rows; ++r) s += dZ[r * cols + c];
    db[c] = s;
}

__global__ void k_adam(float* p, const float* g, float* m1, float* m2, long long n, float lr, float b1, float b2,
                       float c1, float c2, float eps) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const float gg = g[e];
        const float a = b1 * m1[e] + (1.f - b1) * gg;
        const float b = b2 * m2[e] + (1.f - b2) * gg * gg;
        m1[e] = a;
        m2[e] = b;
        p[e] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
    }
}

__global__ void k_gather_rows(const float* src, const int* idx, float* dst, int rows, int cols) {
    const long long n = (long long)rows * cols;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const long long r = e / cols;
        dst[e] = src[(long long)idx[r] * cols + e % cols];
    }
}

// Workspace and one forward/backward pass over `rows` samples.
struct MlpWork {
    int in, out, rows;
    float *Z1, *H1, *Z2, *H2, *Yp, *dY, *dH, *dZ;
    double* loss_partial;
};

static const int EW_BLOCKS = 1024;

// forward (+ backward into grad when grad != null); returns the sum of squared errors via loss_partial
static void forward_backward(const MlpWork& w, const float* P, const float* X, const float* Y, float* grad,
                             float scale, cudaStream_t st) {
    const int H = MLP_HIDDEN, in = w.in, out = w.out, n = w.rows;
    const float* W1 = P;
    const float* b1 = W1 + H * in;
    const float* W2 = b1 + H;
    const float* b2 = W2 + H * H;
    const float* W3 = b2 + H;
    const float* b3 = W3 + out * H;
    gemm(n, H, in, X, in, 0, W1, in, 1, w.Z1, H, 0, st);              // Z1 = X W1^T
    k_bias_act<<<EW_BLOCKS, 256, 0, st>>>(w.Z1, w.H1, b1, n, H);
    gemm(n, H, H, w.H1, H, 0, W2, H, 1, w.Z2, H, 0, st);              // Z2 = H1 W2^T
    k_bias_act<<<EW_BLOCKS, 256, 0, st>>>(w.Z2, w.H2, b2, n, H);
    gemm(n, out, H, w.H2, H, 0, W3, H, 1, w.Yp, out, 0, st);          // Yp = H2 W3^T
    k_bias_act<<<EW_BLOCKS, 256, 0, st>>>(w.Yp, nullptr, b3, n, out);
    k_mse<<<256, 256, 0, st>>>(w.Yp, Y, grad ? w.dY : nullptr, (long long)n * out, scale, w.loss_partial);
    if (!grad) return;
    float* gW1 = grad;
    float* gb1 = gW1 + H * in;
    float* gW2 = gb1 + H;
    float* gb2 = gW2 + H * H;
    float* gW3 = gb2 + H;
    float* gb3 = gW3 + out * H;
    gemm(out, H, n, w.dY, out, 1, w.H2, H, 0, gW3, H, 0, st);         // gW3 = dY^T H2
    k_colsum<<<(out + 127) / 128, 128, 0, st>>>(w.dY, gb3, n, out);
    gemm(n, H, out, w.dY, out, 0, W3, H, 0, w.dH, H, 0, st);          // dH2 = dY W3
    k_gelu_back<<<EW_BLOCKS, 256, 0, st>>>(w.dH, w.Z2, w.dZ, (long long)n * H);
    gemm(H, H, n, w.dZ, H, 1, w.H1, H, 0, gW2, H, 0, st);             // gW2 = dZ2^T H1
    k_colsum<<<1, 128, 0, st>>>(w.dZ, gb2, n, H);
    gemm(n, H, H, w.dZ, H, 0, W2, H, 0, w.dH, H, 0, st);              // dH1 = dZ2 W2
    k_gelu_back<<<EW_BLOCKS, 256, 0, st>>>(w.dH, w.Z1, w.dZ, (long long)n * H);
    gemm(H, in, n, w.dZ, H, 1, X, in, 0, gW1, in, 0, st);             // gW1 = dZ1^T X
    k_colsum<<<1, 128, 0, st>>>(w.dZ, gb1, n, H);
}

static bool alloc_work(MlpWork& w, int in, int out, int rows) {
    const size_t H = MLP_HIDDEN;
    w.in = in;
    w.out = out;
    w.rows = rows;
    float** bufs[] = {&w.Z1, &w.H1, &w.Z2, &w.H2, &w.dH, &w.dZ};
    for (float** b : bufs)
        if (cudaMalloc(b, rows * H * sizeof(float)) != cudaSuccess) return false;
    if (cudaMalloc(&w.Yp, (size_t)rows * out * sizeof(float)) != cudaSuccess) return false;
    if (cudaMalloc(&w.dY, (size_t)rows * out * sizeof(float)) != cudaSuccess) return false;
    return cudaMalloc(&w.loss_partial, 256 * sizeof(double)) == cudaSuccess;
}

static void free_work(MlpWork& w) {
    float* bufs[] = {w.Z1, w.H1, w.Z2, w.H2, w.dH, w.dZ, w.Yp, w.dY};
    for (float* b : bufs)
        if (b) cudaFree(b);
    if (w.loss_partial) cudaFree(w.loss_partial);
}

static double read_loss(const MlpWork& w, cudaStream_t st) {
    double h[256];
    cudaMemcpyAsync(h, w.loss_partial, sizeof(h), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    double s = 0.0;
    for (double v : h) s += v;
    return s;
}

}  // namespace ader

using namespace ader;

extern "C" {

int ader_mlp_shape(int mhd, int* n_in, int* n_hidden, int* n_out, long long* n_params) {
    const int nv = mhd ? 8 : 5;
    if (n_in) *n_in = mlp_in(nv);
    if (n_hidden) *n_hidden = MLP_HIDDEN;
    if (n_out) *n_out = mlp_out(nv);
    if (n_params) *n_params = mlp_params(nv);
    return ADER_OK;
}

int ader_mlp_grad(const float* params, const float* X, const float* Y, long long n, int mhd, float* grad,
                  double* loss_host, void* stream) {
    if (!params || !X || !Y || n <= 0 || n > (1 << 24)) return ADER_ERR_ARG;
    const int nv = mhd ? 8 : 5;
    MlpWork w{};
    cudaStream_t st = (cudaStream_t)stream;
    if (!alloc_work(w, mlp_in(nv), mlp_out(nv), (int)n)) {
        free_work(w);
        return ADER_ERR_CUDA;
    }
    forward_backward(w, params, X, Y, grad, 1.0f / (float)(n * mlp_out(nv)), st);
    const double sse = read_loss(w, st);
    if (loss_host) *loss_host = sse / (double)(n * mlp_out(nv));
    const cudaError_t e = cudaStreamSynchronize(st);
    free_work(w);
    return e == cudaSuccess ? ADER_OK : ADER_ERR_CUDA;
}

int ader_mlp_train(const float* X, const float* Y, long long n, int mhd, int epochs, int batch, float lr,
                   unsigned long long seed, float* params, double* loss_per_epoch_host, void* stream) {
    if (!X || !Y || !params || n < batch || batch <= 0 || epochs <= 0 || !(lr > 0)) return ADER_ERR_ARG;
    const int nv = mhd ? 8 : 5;
    const int in = mlp_in(nv), out = mlp_out(nv);
    const long long np = mlp_params(nv);
    cudaStream_t st = (cudaStream_t)stream;
    MlpWork w{};
    float *grad = nullptr, *m1 = nullptr, *m2 = nullptr, *Xb = nullptr, *Yb = nullptr;
    int* idx_d = nullptr;
    bool ok = alloc_work(w, in, out, batch);
    ok = ok && cudaMalloc(&grad, np * sizeof(float)) == cudaSuccess;
    ok = ok && cudaMalloc(&m1, np * sizeof(float)) == cudaSuccess;
    ok = ok && cudaMalloc(&m2, np * sizeof(float)) == cudaSuccess;
    ok = ok && cudaMalloc(&Xb, (size_t)batch * in * sizeof(float)) == cudaSuccess;
    ok = ok && cudaMalloc(&Yb, (size_t)batch * out * sizeof(float)) == cudaSuccess;
    ok = ok && cudaMalloc(&idx_d, (size_t)n * sizeof(int)) == cudaSuccess;
    int rc = ADER_OK;
    if (!ok) rc = ADER_ERR_CUDA;
    if (rc == ADER_OK) {
        cudaMemsetAsync(m1, 0, np * sizeof(float), st);
        cudaMemsetAsync(m2, 0, np * sizeof(float), st);
        std::vector<int> perm(n);
        unsigned long long s = seed * 6364136223846793005ull + 1442695040888963407ull;
        long long step = 0;
        const long long nb = n / batch;
        for (int ep = 0; ep < epochs && rc == ADER_OK; ++ep) {
            for (long long i = 0; i < n; ++i) perm[i] = (int)i;
            for (long long i = n - 1; i > 0; --i) {     // Fisher-Yates with a 64-bit LCG
                s = s * 6364136223846793005ull + 1442695040888963407ull;
                const long long j = (long long)((s >> 33) % (unsigned long long)(i + 1));
                const int t = perm[i];
                perm[i] = perm[j];
                perm[j] = t;
            }
            cudaMemcpyAsync(idx_d, perm.data(), n * sizeof(int), cudaMemcpyHostToDevice, st);
            double sse = 0.0;
            for (long long b = 0; b < nb; ++b) {
                k_gather_rows<<<EW_BLOCKS, 256, 0, st>>>(X, idx_d + b * batch, Xb, batch, in);
                k_gather_rows<<<EW_BLOCKS, 256, 0, st>>>(Y, idx_d + b * batch, Yb, batch, out);
                forward_backward(w, params, Xb, Yb, grad, 1.0f / (float)((long long)batch * out), st);
                ++step;
                const float c1 = 1.f - powf(0.9f, (float)step), c2 = 1.f - powf(0.999f, (float)step);
                k_adam<<<EW_BLOCKS, 256, 0, st>>>(params, grad, m1, m2, np, lr, 0.9f, 0.999f, c1, c2, 1e-8f);
                if (b == nb - 1 || b % 64 == 0) sse = read_loss(w, st);
            }
            if (loss_per_epoch_host) loss_per_epoch_host[ep] = sse / (double)((long long)batch * out);
            if (cudaGetLastError() != cudaSuccess) rc = ADER_ERR_CUDA;
        }
        if (cudaStreamSynchronize(st) != cudaSuccess) rc = ADER_ERR_CUDA;
    }
    free_work(w);
    void* ptrs[] = {grad, m1, m2, Xb, Yb, idx_d};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    return rc;
}

}  // extern "C"

// Sample generation needs the context internals: defined in api.cu through this hook.
namespace ader {
int launch_guess_samples(const StepArgs& a, const double* U, float* X, float* Y, int* ok, cudaStream_t st) {
    const int T = 128;
    const unsigned blocks = (unsigned)((a.grid.n + T - 1) / T);
    if (a.mhd)
        k_guess_samples<8><<<blocks, T, 0, st>>>(a, U, X, Y, ok);
    else
        k_guess_samples<5><<<blocks, T, 0, st>>>(a, U, X, Y, ok);
    return 1;
}
}  // namespace ader
