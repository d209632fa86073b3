// Batched step: many independent problems of uneven sizes in one launch per
// phase and per variant group (same order, physics, form, solver).
//
// Work layout: the zones of the group's problems are laid end to end, each
// problem padded to a multiple of BATCH_ALIGN zones; zpad[p] is the first
// padded index of problem p (zpad[np] the total).  Launches are persistent:
// a grid sized to the SMs loops over the padded range.  Because every block
// size divides BATCH_ALIGN, all threads of a block always work on the same
// problem, and the padding zones (z >= n of their problem) are skipped.  The
// predictor is the exception: one zone per thread over the whole padded range.
#pragma once
#include "kernels.cuh"
#include "step_kernels.cuh"
#include "weno.cuh"

namespace ader {

constexpr int BATCH_ALIGN = 256;        // block sizes (zones per block) must divide this

struct BatchItem {
    StepArgs a;         // the problem's step arguments (its own scratch, dt_dev and flag)
    double* U;          // state, updated in place
    double* Bf;         // MHD face field, updated in place (null for Euler)
};

// what one launch of a phase over a group needs
struct BatchGroupDev {
    const BatchItem* items;     // device, np entries
    const long long* zpad;      // device, np + 1 entries
    int np;
    long long total;            // zpad[np]
};

ADER_DEV int batch_find(const long long* __restrict__ zpad, int np, long long gz) {
    int lo = 0, hi = np - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (zpad[mid] <= gz)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// The grid-stride walk over the group's padded range: the first padded index of this thread and the
// stride; batch_zone maps a padded index to its problem's item and zone index (false for a padding
// zone).  Every kernel below writes the walk out itself, so that the zone's code is inlined into the
// kernel (a per-zone call through a lambda was compiled as a real call, with the predictor's registers
// spilled around it).
ADER_DEV long long batch_first() { return (long long)blockIdx.x * blockDim.x + threadIdx.x; }
ADER_DEV long long batch_stride() { return (long long)gridDim.x * blockDim.x; }

ADER_DEV bool batch_zone(const BatchGroupDev& g, long long gz, const BatchItem*& it, long long& z) {
    const int p = batch_find(g.zpad, g.np, gz);
    it = g.items + p;
    z = gz - g.zpad[p];
    return z < it->a.grid.n;
}

// One block-iteration's problem for kernels that read the full step arguments: every block covers
// BATCH_ALIGN-aligned zones of one problem, so its item is copied once into shared memory, where the zone
// code reads it (the zone's stores cannot alias it: nothing is reloaded from global memory or held in
// registers across them).  Returns this thread's zone index in that problem (>= its n on padding).
// Called by every thread of the block.
__device__ __forceinline__ long long batch_block_item(const BatchGroupDev& g, long long base, BatchItem& it) {
    static_assert(sizeof(BatchItem) % sizeof(int) == 0, "BatchItem is copied as ints");
    const int p = batch_find(g.zpad, g.np, base);
    __syncthreads();                                    // the previous iteration's readers are done
    for (int w = threadIdx.x; w < (int)(sizeof(BatchItem) / sizeof(int)); w += blockDim.x)
        reinterpret_cast<int*>(&it)[w] = reinterpret_cast<const int*>(g.items + p)[w];
    __syncthreads();
    return base + threadIdx.x - g.zpad[p];
}

template <int ORDER, class R>
__global__ void __launch_bounds__(256) kb_face_b(BatchGroupDev g) {
    for (long long gz = batch_first(); gz < g.total; gz += batch_stride()) {
        const BatchItem* it;
        long long z;
        if (!batch_zone(g, gz, it, z)) continue;
        const Grid gr = it->a.grid;    // local copies: the zone's stores cannot alias them
        zone_face_b<ORDER, R>(gr, it->Bf, (R*)it->a.ZB, (R*)it->a.S1, z);
    }
}

// the FP32 copy of each problem's state (five values per zone), rounded by integer operations
static __global__ void __launch_bounds__(256) kb_to_f32(BatchGroupDev g) {
    for (long long gz = batch_first(); gz < g.total; gz += batch_stride()) {
        const BatchItem* it;
        long long z;
        if (!batch_zone(g, gz, it, z)) continue;
        float* Uf = const_cast<float*>(it->a.Uf);
        const double* U = it->U;
        const long long N = it->a.grid.n;
        double u[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) u[v] = U[v * N + z];
#pragma unroll
        for (int v = 0; v < 5; ++v) Uf[v * N + z] = f32_of_f64(u[v]);
    }
}

template <int ORDER, int NV, class R>
__global__ void __launch_bounds__(128, 5) kb_weno1d(BatchGroupDev g) {
    for (long long gz = batch_first(); gz < g.total; gz += batch_stride()) {
        const BatchItem* it;
        long long z;
        if (!batch_zone(g, gz, it, z)) continue;
        const Grid gr = it->a.grid;
        zone_weno1d<ORDER, NV, R>(gr, it->a.Uf, (const R*)it->a.ZB, (R*)it->a.S1, z);
    }
}

// at most 128 zones per block and three blocks per SM, as the single-problem kernel gets them: at order 4
// the cross moments need about 170 registers, and with 256-thread blocks only one block fits an SM
template <int ORDER, int NV, class R>
__global__ void __launch_bounds__(128, 3) kb_cross1(BatchGroupDev g) {
    for (long long gz = batch_first(); gz < g.total; gz += batch_stride()) {
        const BatchItem* it;
        long long z;
        if (!batch_zone(g, gz, it, z)) continue;
        const Grid gr = it->a.grid;
        zone_cross1<ORDER, NV, R>(gr, (const R*)it->a.S1, (R*)it->a.S2, z);
    }
}

template <int NV, class R>
__global__ void __launch_bounds__(256) kb_cross2(BatchGroupDev g) {
    for (long long gz = batch_first(); gz < g.total; gz += batch_stride()) {
        const BatchItem* it;
        long long z;
        if (!batch_zone(g, gz, it, z)) continue;
        const Grid gr = it->a.grid;
        zone_cross2<NV, R>(gr, (R*)it->a.S2, z);
    }
}

// at most 128 zones per block, three blocks per SM (two at order 4 and for MHD at order 3), as the
// single-problem FP32 predictor
constexpr int BATCH_PREDICT_MAX_THREADS = 128;

// One zone per thread (never persistent): a grid-stride loop around the predictor's body keeps a few
// more values live through it, and at 168 registers those spill (about 1 KB more local traffic per zone
// at order 3); the launch covers the padded range (batch_phase_persistent).
template <int ORDER, int FORM, int NV, class R>
__global__ void __launch_bounds__(BATCH_PREDICT_MAX_THREADS, ORDER == 4 || (ORDER == 3 && NV == 8) ? 2 : 3)
    kb_predict_faces(BatchGroupDev g) {
    __shared__ BatchItem it;                            // the block's arguments (batch_block_item)
    const long long base = (long long)blockIdx.x * blockDim.x;
    if (base >= g.total) return;                        // the whole block
    const long long z = batch_block_item(g, base, it);
    if (z >= it.a.grid.n) return;
    zone_predict_faces<ORDER, FORM, NV, R>(it.a, it.U, z);
}

// U += dt L(U) in place, dt from the problem's dt_dev: both faces of each direction solved per zone, the
// differences carried in FP32 pairs and only the accumulation in FP64 (zone_flux_update_pair)
template <int SOLVER, int NV, class R>
__global__ void __launch_bounds__(256) kb_flux_update(BatchGroupDev g) {
    __shared__ BatchItem it;
    for (long long base = (long long)blockIdx.x * blockDim.x; base < g.total; base += batch_stride()) {
        const long long z = batch_block_item(g, base, it);
        if (z >= it.a.grid.n) continue;
        double* U = it.U;
        if constexpr (sizeof(R) == 4)
            zone_flux_update_pair<SOLVER, NV>(it.a, U, U, 1.0, 1, z);
        else
            zone_flux_update<SOLVER, NV, R>(it.a, U, U, 1.0, 1, z);
    }
}

template <class R>
__global__ void __launch_bounds__(256) kb_emf(BatchGroupDev g) {
    __shared__ BatchItem it;
    for (long long base = (long long)blockIdx.x * blockDim.x; base < g.total; base += batch_stride()) {
        const long long z = batch_block_item(g, base, it);
        if (z >= it.a.grid.n) continue;
        zone_emf<R>(it.a, z);
    }
}

template <class R>
__global__ void __launch_bounds__(256) kb_ct(BatchGroupDev g) {
    __shared__ BatchItem it;
    for (long long base = (long long)blockIdx.x * blockDim.x; base < g.total; base += batch_stride()) {
        const long long z = batch_block_item(g, base, it);
        if (z >= it.a.grid.n) continue;
        zone_ct<R>(it.a, it.Bf, 1.0, 1, z);
    }
}

// Phases of one step, in order; a group runs those that apply to it.
enum BatchPhase { PH_TO_F32 = 0, PH_FACE_B, PH_WENO1D, PH_CROSS1, PH_CROSS2, PH_PREDICT, PH_UPDATE, PH_EMF, PH_CT,
                  PH_COUNT };

// whether a phase's kernel walks the group's range with a grid-stride loop (any grid size), or needs a
// thread for every padded zone
inline bool batch_phase_persistent(int ph) { return ph != PH_PREDICT; }

// the largest block a phase's kernel is compiled for (its launch bounds)
inline int batch_phase_max_threads(int ph) {
    return ph == PH_PREDICT ? BATCH_PREDICT_MAX_THREADS : (ph == PH_WENO1D || ph == PH_CROSS1) ? 128 : 256;
}

inline bool batch_phase_applies(int ph, int order, int mhd) {
    switch (ph) {
        case PH_FACE_B: return mhd != 0;
        case PH_CROSS1: return order >= 3;
        case PH_CROSS2: return order == 4;
        case PH_EMF:
        case PH_CT: return mhd != 0;
        default: return true;
    }
}

// Launches phase ph of a group of (ORDER, NV) problems with `threads` zones per
// block and `blocks` blocks; returns the kernel (for occupancy queries) through
// *fn when launch is false.  Instantiated per (ORDER, NV) in batch_o*_*.cu (FP32 bulk).
template <int ORDER, int NV>
int batch_phase(int ph, const BatchGroupDev& g, int form, int solver, int threads, int blocks, cudaStream_t st,
                bool launch, const void** fn);

}  // namespace ader
