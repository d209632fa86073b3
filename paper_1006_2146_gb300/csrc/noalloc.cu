// ader_max_dt_static: the CFL time-step reduction without any allocation.
//
// Some callers cannot call cudaMalloc: code that runs inside a stream capture
// or a CUDA-graph node set up by someone else, real-time loops whose memory
// budget is fixed up front, or hosts that forbid device allocation after start
// up.  This entry point needs no context (ader_create allocates) and keeps its
// scratch in a file-scope __device__ array instead: one partial maximum per
// block plus a finished-block counter.
//
// The array lives in every device that loads the library until the process
// exits.  Its size caps the grid at ADER_STATIC_MAX_ZONES zones; larger grids
// are rejected.  The device address of the array is looked up once per device
// (cudaGetSymbolAddress, with that device current) on the first call made on
// it; that first call should therefore come before any stream capture.  All
// calls share the array, so calls that overlap on the GPU (two streams, two
// threads) race and must be serialised by the caller.  The counter is zero
// when the module loads (a __device__ variable starts zeroed) and the last
// block of each call clears it again, so set-up issues no device work.
//
// A zone with rho <= 0, P <= 0 or a value that is not finite has no signal
// speed: the call then writes a quiet NaN as dt, so a step taken with it
// turns the state non-finite, which ader_sync_status reports.
#include <mutex>

#include "../../include/ader.h"
#include "common.cuh"

namespace ader {

constexpr int STATIC_THREADS = 256;
constexpr int STATIC_ZONES_PER_THREAD = 16;
constexpr long long STATIC_ZONES_PER_BLOCK = (long long)STATIC_THREADS * STATIC_ZONES_PER_THREAD;
constexpr int STATIC_MAX_BLOCKS = 65536;

struct StaticScratch {
    double partial[STATIC_MAX_BLOCKS];   // one maximum per block
    unsigned int done;                   // blocks finished in the current call
};

static __device__ __align__(256) StaticScratch g_dt_scratch;

// Same per-zone signal speed and warp-shuffle block maximum as k_max_dt; each
// block owns a fixed chunk of zones and stores its maximum; the last block to
// finish reduces the partials in a fixed order and writes dt.
__global__ void __launch_bounds__(STATIC_THREADS) k_max_dt_static(Grid g, const double* __restrict__ U, double gamma,
                                                                  double idx, double idy, double idz, double cfl,
                                                                  double* dt_out, StaticScratch* scr) {
    const long long N = g.n;
    const long long base = (long long)blockIdx.x * STATIC_ZONES_PER_BLOCK;
    double s = 0.0;
    bool bad = false;
    for (int r = 0; r < STATIC_ZONES_PER_THREAD; ++r) {
        const long long z = base + (long long)r * STATIC_THREADS + threadIdx.x;
        if (z >= N) break;
        const double rho = U[z], mx = U[N + z], my = U[2 * N + z], mz = U[3 * N + z], E = U[4 * N + z];
        const double ir = 1.0 / rho;
        const double vx = mx * ir, vy = my * ir, vz = mz * ir;
        const double p = (gamma - 1.0) * (E - 0.5 * (mx * vx + my * vy + mz * vz));
        if (!(rho > 0.0) || !(p > 0.0) || !isfinite(p) || !isfinite(vx + vy + vz)) {
            bad = true;
            continue;
        }
        const double a = sqrt(gamma * p * ir);
        s = fmax(s, (fabs(vx) + a) * idx + (fabs(vy) + a) * idy + (fabs(vz) + a) * idz);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
    __shared__ double warp_max[STATIC_THREADS / 32];
    __shared__ bool last;
    if ((threadIdx.x & 31) == 0) warp_max[threadIdx.x >> 5] = s;
    // a block that met a non-physical zone stores -1 (speeds are never negative)
    const bool block_bad = __syncthreads_or(bad) != 0;
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int w = 0; w < STATIC_THREADS / 32; ++w) b = fmax(b, warp_max[w]);
        scr->partial[blockIdx.x] = block_bad ? -1.0 : b;
        __threadfence();
        last = (atomicAdd(&scr->done, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double m = 0.0;
    bool any_bad = false;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += STATIC_THREADS) {
        const double v = ((volatile double*)scr->partial)[b];
        any_bad |= v < 0.0;
        m = fmax(m, v);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) warp_max[threadIdx.x >> 5] = m;
    any_bad = __syncthreads_or(any_bad) != 0;
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int w = 0; w < STATIC_THREADS / 32; ++w) b = fmax(b, warp_max[w]);
        *dt_out = any_bad ? __longlong_as_double(0x7ff8000000000000LL) : (b > 0.0 ? cfl / b : 0.0);
        scr->done = 0u;
    }
}

}  // namespace ader

namespace {
constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mutex;
ader::StaticScratch* g_scratch_ptr[MAX_DEVICES] = {};
}  // namespace

extern "C" int ader_max_dt_static(const ader_grid* g, double gamma, const double* U, double cfl, double* dt_dev,
                                  void* stream) {
    using namespace ader;
    if (!g || !U || !dt_dev || g->nx < 1 || g->ny < 1 || g->nz < 1) return ADER_ERR_ARG;
    if (!(g->dx > 0) || !(g->dy > 0) || !(g->dz > 0) || !(gamma > 1.0) || !(cfl > 0.0)) return ADER_ERR_ARG;
    const long long n = (long long)g->nx * g->ny * g->nz;
    if (n > ADER_STATIC_MAX_ZONES) return ADER_ERR_ARG;          // beyond the static scratch
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return ADER_ERR_CUDA;
    StaticScratch* scr = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_ptr[dev]) {
            // set-up on this device: the device address of the array (its counter starts at zero)
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_dt_scratch) != cudaSuccess || !p) return ADER_ERR_CUDA;
            g_scratch_ptr[dev] = (StaticScratch*)p;
        }
        scr = g_scratch_ptr[dev];
    }
    const Grid grid{g->nx, g->ny, g->nz, n};
    const unsigned blocks = (unsigned)((n + STATIC_ZONES_PER_BLOCK - 1) / STATIC_ZONES_PER_BLOCK);
    k_max_dt_static<<<blocks, STATIC_THREADS, 0, (cudaStream_t)stream>>>(grid, U, gamma, 1.0 / g->dx, 1.0 / g->dy,
                                                                         1.0 / g->dz, cfl, dt_dev, scr);
    return cudaGetLastError() == cudaSuccess ? ADER_OK : ADER_ERR_CUDA;
}
