// Learned predictor guess on the 5th-generation tensor cores (tcgen05).
//
// One CTA per SM runs GROUPS independent pipelines of 128 threads, each over
// tiles of 128 zones (persistent over the grid); the FP16 weights in shared
// memory serve all of them.  In a pipeline each thread computes its zone's
// features (mlp.cuh) and writes them as FP16 into the group's A operand; one
// thread issues the three layers as tcgen05.mma (kind::f16, M = 128, FP32
// accumulator in the group's 128 TMEM columns); after each layer every warp
// reads its 32 accumulator lanes back with tcgen05.ld, adds the bias, applies
// GELU (tanh form, hardware tanh, packed FP16 pairs) and writes the next A operand.  The groups
// synchronise on their own named barriers, so while one waits on memory or on
// its MMAs the others compute.
//
// Operand layout: K-major, no swizzle.  A tile of R rows and K columns is
// stored as 8 x 8 "core matrices" (8 rows of 16 bytes, 128 contiguous bytes);
// core matrix (row group rg, column chunk kc) sits at byte
// (rg * K/8 + kc) * 128, so the descriptor's leading byte offset (next chunk
// along K) is 128 and its stride byte offset (next 8-row group) is K/8 * 128.
//
// Every wait on the MMA barrier is bounded: on time-out the CTA raises
// FLAG_TIMEOUT, waits once more (bounded) for its MMAs, frees its TMEM and
// returns.  A launch armed by ader_test_bounded_wait (a.wait_test) issues no
// MMA and commits nothing for its first layer, so that nothing ever arrives
// on the barrier; its waits then run out after WAIT_TEST_LIMIT tries (with no
// MMA in flight, the clean-up wait has nothing to wait for either) and the
// time-out path above runs for real.
#include <cuda_fp16.h>

#include "kernels.cuh"
#include "mlp.cuh"
#include "step_kernels.cuh"

namespace ader {
namespace {

constexpr int TM = 128;                  // zones per tile = MMA M = TMEM lanes = threads per group
constexpr int GROUPS = 4;                // pipelines per CTA (512 threads)
constexpr unsigned TMEM_COLS = 128;      // accumulator columns per group: the widest layer
constexpr long long WAIT_LIMIT = 1ll << 22;
constexpr long long WAIT_TEST_LIMIT = 1024;

__host__ __device__ constexpr int k1pad(int nv) { return (mlp_in(nv) + 15) / 16 * 16; }
__host__ __device__ constexpr int n3pad(int nv) { return (mlp_out(nv) + 15) / 16 * 16; }

template <int NV>
struct TcSmem {
    static constexpr int H = MLP_HIDDEN, K1 = k1pad(NV), N3 = n3pad(NV);
    __half W1[H * K1];      // B of layer 1: H rows (outputs) x K1
    __half W2[H * H];       // B of layer 2
    __half W3[N3 * H];      // B of layer 3: N3 rows x H
    __half A[GROUPS][TM * H];   // per group A: features (TM x K1), then the hidden layers (TM x H)
    float b1[H], b2[H], b3[N3];
    unsigned long long mbar[GROUPS];
    unsigned tmem_base;
};

// element offset of (row r, column k) in a K-major core-matrix tile with K columns
__device__ __forceinline__ int koff(int r, int k, int K) {
    return (((r >> 3) * (K >> 3) + (k >> 3)) * 8 + (r & 7)) * 8 + (k & 7);
}

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t sdesc(const void* p, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr(p) >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);     // no swizzle
}

// instruction descriptor of kind::f16: D FP32, A and B FP16, both K-major
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N) {
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(id), "r"(acc));
}

__device__ __forceinline__ void mma_commit(unsigned long long* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(unsigned long long* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(saddr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, uint32_t parity, long long limit) {
    for (long long i = 0; i < limit; ++i)
        if (mbar_try(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 consecutive accumulator columns of this thread's lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// GELU, tanh form, on two FP16 values at once: 0.5 x (1 + tanh(x (c0 + c1 x^2)))
// with c0 = sqrt(2/pi), c1 = 0.044715 c0, and the hardware tanh.  The result
// feeds the next layer as an FP16 operand, so computing it in FP16 costs
// about one rounding of that operand; the packed form halves the epilogue's
// instructions, which bound this kernel.
__device__ __forceinline__ __half2 gelu_h2(__half2 x) {
    const __half2 c0 = __float2half2_rn(0.7978845608028654f);
    const __half2 c1 = __float2half2_rn(0.044715f * 0.7978845608028654f);
    const __half2 half = __float2half2_rn(0.5f);
    const __half2 u = __hmul2(x, __hfma2(c1, __hmul2(x, x), c0));
    uint32_t ui = *reinterpret_cast<const uint32_t*>(&u), ti;
    asm("tanh.approx.f16x2 %0, %1;" : "=r"(ti) : "r"(ui));
    const __half2 t = *reinterpret_cast<const __half2*>(&ti);
    const __half2 hx = __hmul2(half, x);
    return __hfma2(hx, t, hx);
}

// the K steps of one layer: D[tmem] = A (TM x K) * B^T (N x K)
__device__ __forceinline__ void issue_layer(uint32_t tmem, const __half* A, const __half* B, int K, int N) {
    const uint32_t sbo = (uint32_t)(K / 8) * 128u;
    const uint32_t id = idesc_f16(TM, N);
    for (int ks = 0; ks < K / 16; ++ks)
        mma_f16(tmem, sdesc(A + ks * 128, 128u, sbo), sdesc(B + ks * 128, 128u, sbo), id, ks > 0 ? 1u : 0u);
}

// accumulator + bias -> GELU -> FP16 into the A operand (K = H) at this thread's row
__device__ __forceinline__ void hidden_epilogue(__half* A, const float* bias, uint32_t tlane, int row) {
    constexpr int H = MLP_HIDDEN;
#pragma unroll 1
    for (int c = 0; c < H; c += 16) {
        float v[16];
        tmem_ld16(tlane + (uint32_t)c, v);
        __align__(16) __half2 h[8];
#pragma unroll
        for (int j = 0; j < 8; ++j)
            h[j] = gelu_h2(__floats2half2_rn(v[2 * j] + bias[c + 2 * j], v[2 * j + 1] + bias[c + 2 * j + 1]));
        *reinterpret_cast<uint4*>(&A[koff(row, c, H)]) = *reinterpret_cast<const uint4*>(&h[0]);
        *reinterpret_cast<uint4*>(&A[koff(row, c + 8, H)]) = *reinterpret_cast<const uint4*>(&h[4]);
    }
}

// named barrier of one group (ids 1..GROUPS; 0 is __syncthreads)
__device__ __forceinline__ void group_sync(int id) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(TM) : "memory"); }

// the same barrier, returning whether any thread of the group passed true
__device__ __forceinline__ bool group_sync_or(int id, bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(r)
        : "r"(v ? 1u : 0u), "r"(id), "r"(TM)
        : "memory");
    return r != 0;
}

template <int NV, class R>
__global__ void __launch_bounds__(TM * GROUPS, 1) k_guess_tc(StepArgs a, const double* __restrict__ U) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((1024u - (saddr(smem_raw) & 1023u)) & 1023u);   // 1 KB aligned
    TcSmem<NV>& s = *reinterpret_cast<TcSmem<NV>*>(base);
    constexpr int IN = mlp_in(NV), OUT = mlp_out(NV), H = MLP_HIDDEN, K1 = k1pad(NV), N3 = n3pad(NV);
    constexpr int NT = TM * GROUPS;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int g = tid / TM, row = tid % TM;          // pipeline and its tile row

    // weights -> FP16 operand layout, biases -> FP32 (all pipelines share them)
    const float* W1 = a.guess;
    const float* b1 = W1 + H * IN;
    const float* W2 = b1 + H;
    const float* b2 = W2 + H * H;
    const float* W3 = b2 + H;
    const float* b3 = W3 + OUT * H;
    for (int e = tid; e < H * K1; e += NT) {
        const int r = e / K1, k = e % K1;
        s.W1[koff(r, k, K1)] = __float2half_rn(k < IN ? W1[r * IN + k] : 0.f);
    }
    for (int e = tid; e < H * H; e += NT) s.W2[koff(e / H, e % H, H)] = __float2half_rn(W2[e]);
    for (int e = tid; e < N3 * H; e += NT) {
        const int r = e / H, k = e % H;
        s.W3[koff(r, k, H)] = __float2half_rn(r < OUT ? W3[r * H + k] : 0.f);
    }
    for (int e = tid; e < H; e += NT) {
        s.b1[e] = b1[e];
        s.b2[e] = b2[e];
    }
    for (int e = tid; e < N3; e += NT) s.b3[e] = e < OUT ? b3[e] : 0.f;
    if (tid < GROUPS) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&s.mbar[tid])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&s.tmem_base)),
                     "r"(TMEM_COLS * GROUPS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tbase = s.tmem_base + (uint32_t)(g * TMEM_COLS);            // the group's columns
    const uint32_t tlane = tbase + ((uint32_t)((warp & 3) * 32) << 16);        // this warp's 32 lanes
    __half* A = s.A[g];
    unsigned long long* bar = &s.mbar[g];
    const int bid = 1 + g;

    const double dt = a.dt_dev ? *a.dt_dev : a.dt;
    const float cx = (float)(dt * a.idx[0]), cy = (float)(dt * a.idx[1]), cz = (float)(dt * a.idx[2]);
    const long long N = a.grid.n;
    const long long cnt = *a.Gcount;                  // the zones with slopes (k_guess_compact)
    const long long ntiles = (cnt + TM - 1) / TM;
    uint32_t parity = 0;
    bool timed_out = false;
    const bool test = a.wait_test != 0;
    const long long limit = test ? WAIT_TEST_LIMIT : WAIT_LIMIT;
    auto sync_mma = [&]() -> bool {          // the group waits for its committed layer
        const bool ok = mbar_wait(bar, parity, limit);
        parity ^= 1u;
        fence_after();
        return !group_sync_or(bid, !ok);
    };
    auto handoff = [&]() {                   // A written by the group -> visible to its MMAs
        fence_async_smem();
        fence_before();
        group_sync(bid);
        fence_after();
    };
    for (long long t = (long long)blockIdx.x * GROUPS + g; t < ntiles; t += (long long)gridDim.x * GROUPS) {
        const long long z = t * TM + row < cnt ? (long long)a.Glist[t * TM + row] : -1;
        float sv[NV] = {};
        bool act = false;
        {
            float x[K1];
#pragma unroll
            for (int k = 0; k < K1; ++k) x[k] = 0.f;
            if (z >= 0) {
                Vec<NV, R> m[11];
                load_modes<3>(a, U, z, m);
                const float mag = guess_features_f32<NV, R>(m, cx, cy, cz, x, sv);
                act = mag > (float)GUESS_MAG_MIN;
            }
            if (!act) {
#pragma unroll
                for (int k = 0; k < K1; ++k) x[k] = 0.f;
            }
#pragma unroll
            for (int kc = 0; kc < K1; kc += 8) {
                __align__(16) __half h[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) h[j] = __float2half_rn(x[kc + j]);
                *reinterpret_cast<uint4*>(&A[koff(row, kc, K1)]) = *reinterpret_cast<const uint4*>(h);
            }
        }
        // layer 1 (none in a test of the bounded waits: the barrier then never completes)
        handoff();
        if (row == 0 && !test) {
            issue_layer(tbase, A, s.W1, K1, H);
            mma_commit(bar);
        }
        if (!sync_mma()) { timed_out = true; break; }
        hidden_epilogue(A, s.b1, tlane, row);
        // layer 2
        handoff();
        if (row == 0) {
            issue_layer(tbase, A, s.W2, H, H);
            mma_commit(bar);
        }
        if (!sync_mma()) { timed_out = true; break; }
        hidden_epilogue(A, s.b2, tlane, row);
        // layer 3
        handoff();
        if (row == 0) {
            issue_layer(tbase, A, s.W3, H, N3);
            mma_commit(bar);
        }
        if (!sync_mma()) { timed_out = true; break; }
#pragma unroll
        for (int c = 0; c < N3; c += 16) {
            float v[16];
            tmem_ld16(tlane + (uint32_t)c, v);
            if (z >= 0) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int o = c + j;
                    if (o < OUT) a.G[(long long)o * N + z] = act ? (v[j] + s.b3[o]) * sv[o % NV] : 0.f;
                }
            }
        }
        fence_before();
        group_sync(bid);         // the next tile's layer 1 overwrites A and the accumulator
        fence_after();
    }
    if (timed_out) {
        if (row == 0) raise_flag(a.flag, FLAG_TIMEOUT);
        mbar_wait(bar, parity ^ 1u, limit);  // bounded: let the group's MMAs in flight finish before TMEM is freed
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s.tmem_base),
                     "r"(TMEM_COLS * GROUPS)
                     : "memory");
}

// The zones whose guess is not exactly zero: a zone runs the network only when its slope magnitude g
// exceeds GUESS_MAG_MIN (below it the guess is zero by definition).  Each zone writes its flag; the
// zones with slopes get a slot in the list (warp-aggregated atomics: the order of the list is not
// fixed, each zone's guess is its own).  Gzero (non-null for ader_guess_eval) receives the zero guess of
// every other zone; the step's predictor reads the flag instead.
template <int NV, class R>
__global__ void __launch_bounds__(256) k_guess_compact(StepArgs a, const double* __restrict__ U, float* Gzero) {
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    bool act = false;
    if (z < a.grid.n) {
        Vec<NV, R> m[11];
        load_modes<3>(a, U, z, m);
        act = guess_mag_f32<NV, R>(m) > (float)GUESS_MAG_MIN;
        a.Gact[z] = act ? 1 : 0;
        if (!act && Gzero) {
#pragma unroll
            for (int o = 0; o < 5 * NV; ++o) Gzero[(long long)o * a.grid.n + z] = 0.f;
        }
    }
    const unsigned ballot = __ballot_sync(0xffffffffu, act);
    if (ballot == 0u) return;
    const int lane = threadIdx.x & 31;
    unsigned base = 0;
    if (lane == __ffs(ballot) - 1) base = atomicAdd(a.Gcount, (unsigned)__popc(ballot));
    base = __shfl_sync(0xffffffffu, base, __ffs(ballot) - 1);
    if (act) a.Glist[base + __popc(ballot & ((1u << lane) - 1u))] = (int)z;
}

template <int NV, class R>
int launch_nv(const StepArgs& a, const double* U, cudaStream_t st, float* Gzero) {
    static int max_blocks_dev[64] = {};     // per instantiation and device: resident CTAs per SM x SMs
    const size_t smem = sizeof(TcSmem<NV>) + 1024;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur < 0 || cur >= 64) return -1;
    int& max_blocks = max_blocks_dev[cur];
    if (max_blocks == 0) {
        if (cudaFuncSetAttribute(k_guess_tc<NV, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return -1;
        // all of the SM's unified L1/shared storage as shared memory: two CTAs (two tiles) per SM
        if (cudaFuncSetAttribute(k_guess_tc<NV, R>, cudaFuncAttributePreferredSharedMemoryCarveout, 100) !=
            cudaSuccess)
            return -1;
        int dev = 0, sms = 0, smem_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        // one CTA per SM: its GROUPS pipelines hold all 512 TMEM columns
        (void)smem_sm;
        max_blocks = sms;
    }
    if (cudaMemsetAsync(a.Gcount, 0, sizeof(unsigned), st) != cudaSuccess) return -1;
    k_guess_compact<NV, R><<<(unsigned)((a.grid.n + 255) / 256), 256, 0, st>>>(a, U, Gzero);
    // the count lives on the device: one persistent CTA per SM walks the list's tiles
    const long long tiles = (a.grid.n + TM - 1) / TM;
    const long long want = (tiles + GROUPS - 1) / GROUPS;
    const unsigned blocks = (unsigned)(want < max_blocks ? want : max_blocks);
    k_guess_tc<NV, R><<<blocks, TM * GROUPS, smem, st>>>(a, U);
    return 2;
}

}  // namespace

template <class R>
int launch_guess(const StepArgs& a, const double* U, cudaStream_t st, float* Gzero) {
    return a.mhd ? launch_nv<8, R>(a, U, st, Gzero) : launch_nv<5, R>(a, U, st, Gzero);
}

template int launch_guess<double>(const StepArgs&, const double*, cudaStream_t, float*);
template int launch_guess<float>(const StepArgs&, const double*, cudaStream_t, float*);

}  // namespace ader
