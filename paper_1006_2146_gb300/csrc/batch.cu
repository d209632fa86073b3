// The batched C ABI (ader_batch_*): many independent problems stepped
// together, FP32 bulk with FP64 update and reductions.
//
// One step = the per-problem CFL dt (one launch over every problem, block
// reductions into a per-problem maximum, then one finishing launch), then for
// every variant group (same order, physics, form and solver) its phases, each
// one persistent launch over all of the group's problems.  The groups run on
// their own streams, forked from and joined to the caller's stream, so small
// groups fill the GPU together.  The whole step is captured once into a CUDA
// graph and replayed; a change of the state pointers, dt buffer or CFL number
// captures it again.  ader_batch_tune times each (group, phase) over a few
// block sizes and persistent grid sizes on copies of the state and keeps the
// fastest.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/ader.h"
#include "batch.cuh"

namespace ader {

// ---------------------------------------------------------------- per-problem CFL dt
// Every block works on one problem (padded layout, 256 zones per block and
// iteration); its maximum goes to smax[p] as the bit pattern of a
// non-negative double, which orders like an unsigned integer.  Every batched
// problem is FP32 bulk: each zone's signal speed is FP32 from the state rounded
// by integer operations, with the FP32 copies of gamma and 1/dx (no FP64
// division or conversion per zone), as the single-problem FP32 reduction; the
// block's maximum is widened to FP64 exactly.
__global__ void __launch_bounds__(256) kb_max_dt(BatchGroupDev g, unsigned long long* smax) {
    __shared__ float wm[8];
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long base = (long long)blockIdx.x * blockDim.x; base < g.total; base += stride) {
        const long long gz = base + threadIdx.x;
        const int p = batch_find(g.zpad, g.np, base);          // the same for the whole block
        const BatchItem& it = g.items[p];
        const Grid gr = it.a.grid;
        const long long z = gz - g.zpad[p];
        float s = 0.f;
        if (z < gr.n) {
            using F = float;
            const long long N = gr.n;
            const double* U = it.U;
            const F gamma = it.a.gamma_f;
            const F ix = it.a.idx_f[0], iy = it.a.idx_f[1], iz = it.a.idx_f[2];
            const F rho = f32_of_f64(U[z]), mx = f32_of_f64(U[N + z]), my = f32_of_f64(U[2 * N + z]),
                    mz = f32_of_f64(U[3 * N + z]), E = f32_of_f64(U[4 * N + z]);
            const F ir = F(1) / rho;
            const F vx = mx * ir, vy = my * ir, vz = mz * ir;
            bool bad;
            if (it.Bf) {
                int i, j, k;
                zone_ijk(gr, z, i, j, k);
                const double* Bf = it.Bf;
                Vec<8, F> u;
                u[0] = rho; u[1] = mx; u[2] = my; u[3] = mz; u[4] = E;
                u[5] = F(0.5 * (Bf[z] + Bf[nbr(gr, i, j, k, 1, 0, 0)]));
                u[6] = F(0.5 * (Bf[N + z] + Bf[N + nbr(gr, i, j, k, 0, 1, 0)]));
                u[7] = F(0.5 * (Bf[2 * N + z] + Bf[2 * N + nbr(gr, i, j, k, 0, 0, 1)]));
                const Prim<8, F> q = primitives(u, gamma - F(1));
                bad = !(rho > F(0)) || !(q.p > F(0));
                if (!bad)
                    s = (fabsf(vx) + fast_speed<0>(u, q, gamma)) * ix + (fabsf(vy) + fast_speed<1>(u, q, gamma)) * iy +
                        (fabsf(vz) + fast_speed<2>(u, q, gamma)) * iz;
            } else {
                const F pr = (gamma - F(1)) * (E - F(0.5) * (mx * vx + my * vy + mz * vz));
                bad = !(rho > F(0)) || !(pr > F(0));
                if (!bad) {
                    const F a = sqrtf(gamma * pr * ir);
                    s = (fabsf(vx) + a) * ix + (fabsf(vy) + a) * iy + (fabsf(vz) + a) * iz;
                }
            }
            if (bad) raise_flag(it.a.flag, FLAG_UNPHYSICAL);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s = fmaxf(s, __shfl_xor_sync(0xffffffffu, s, o));
        if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            float b = 0.f;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b = fmaxf(b, wm[w]);
            atomicMax(&smax[p], (unsigned long long)__double_as_longlong(f64_of_f32(b)));
        }
        __syncthreads();
    }
}

// dt[p] = cfl / smax[p] (0 when the maximum is 0); clears smax for the next step
__global__ void kb_max_dt_finish(int np, double cfl, unsigned long long* smax, double* dt) {
    for (int p = threadIdx.x; p < np; p += blockDim.x) {
        const double m = __longlong_as_double((long long)smax[p]);
        dt[p] = m > 0.0 ? cfl / m : 0.0;
        smax[p] = 0ull;
    }
}

}  // namespace ader

using namespace ader;

namespace {

struct Tuned {
    int threads = 128;
    int blocks = 0;         // 0: one block per 'threads' zones (not persistent)
    float ms = -1.f;        // measured time of the choice (-1: not tuned)
};

struct Group {
    int order, mhd, form, solver;
    std::vector<int> members;               // problem indices
    BatchItem* items_dev = nullptr;
    long long* zpad_dev = nullptr;
    long long total = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    Tuned tuned[PH_COUNT];
};

}  // namespace

struct ader_batch {
    int n = 0;
    int sms = 0;
    std::vector<ader_grid> grids;
    std::vector<int> order, solver, mhd, form;
    std::vector<double> gamma;
    std::vector<long long> zones;
    std::vector<BatchItem> items;           // host copies (pointers filled per state)
    void* arena = nullptr;                  // all problems' scratch
    unsigned* flags = nullptr;              // one error word per problem
    double* dt_int = nullptr;               // per-problem dt (device), when the caller passes none
    unsigned long long* smax = nullptr;     // per-problem running maximum of the dt reduction
    BatchItem* all_items_dev = nullptr;     // every problem, for the dt reduction
    long long* all_zpad_dev = nullptr;
    long long all_total = 0;
    std::vector<Group> groups;
    cudaEvent_t fork = nullptr;
    // the legacy default stream cannot be captured: steps called on it run on `own`, ordered by two events
    cudaStream_t own = nullptr;
    cudaEvent_t bridge_in = nullptr, bridge_out = nullptr;
    // captured step
    cudaGraphExec_t exec = nullptr;
    std::vector<const void*> key;           // pointers and mode the graph was captured with
    double key_cfl = 0.0;
    bool tuned = false;
    std::string err;
};

namespace {

int fail(ader_batch* b, int code, const std::string& msg) {
    if (b) b->err = msg;
    return code;
}

int cuda_ok(ader_batch* b, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return ADER_OK;
    return fail(b, ADER_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

template <int O>
int phase_nv(int nv, int ph, const BatchGroupDev& g, int form, int solver, int T, int B, cudaStream_t st, bool go,
             const void** fn) {
    return nv == 8 ? batch_phase<O, 8>(ph, g, form, solver, T, B, st, go, fn)
                   : batch_phase<O, 5>(ph, g, form, solver, T, B, st, go, fn);
}

int run_phase(const Group& gr, int ph, int T, int B, cudaStream_t st, bool go, const void** fn) {
    BatchGroupDev g{gr.items_dev, gr.zpad_dev, (int)gr.members.size(), gr.total};
    const int nv = gr.mhd ? 8 : 5;
    if (B <= 0 || !batch_phase_persistent(ph)) B = (int)std::max<long long>(1, (gr.total + T - 1) / T);
    switch (gr.order) {
        case 2: return phase_nv<2>(nv, ph, g, gr.form, gr.solver, T, B, st, go, fn);
        case 3: return phase_nv<3>(nv, ph, g, gr.form, gr.solver, T, B, st, go, fn);
        default: return phase_nv<4>(nv, ph, g, gr.form, gr.solver, T, B, st, go, fn);
    }
}

// Uploads the items (state pointers set) and padded offsets of every group and of the whole batch.
int upload(ader_batch* b, double* const* U, double* const* Bf, const double* dt_dev) {
    for (int p = 0; p < b->n; ++p) {
        b->items[p].U = U[p];
        b->items[p].Bf = b->mhd[p] ? Bf[p] : nullptr;
        b->items[p].a.Bface = b->items[p].Bf;
        b->items[p].a.dt_dev = (dt_dev ? dt_dev : b->dt_int) + p;
    }
    std::vector<long long> zp(b->n + 1, 0);
    for (int p = 0; p < b->n; ++p)
        zp[p + 1] = zp[p] + (b->zones[p] + BATCH_ALIGN - 1) / BATCH_ALIGN * BATCH_ALIGN;
    b->all_total = zp[b->n];
    if (int rc = cuda_ok(b, cudaMemcpy(b->all_items_dev, b->items.data(), b->n * sizeof(BatchItem),
                                       cudaMemcpyHostToDevice), "upload items"))
        return rc;
    if (int rc = cuda_ok(b, cudaMemcpy(b->all_zpad_dev, zp.data(), (b->n + 1) * sizeof(long long),
                                       cudaMemcpyHostToDevice), "upload offsets"))
        return rc;
    for (auto& g : b->groups) {
        std::vector<BatchItem> it;
        std::vector<long long> gz(1, 0);
        for (int p : g.members) {
            it.push_back(b->items[p]);
            gz.push_back(gz.back() + (b->zones[p] + BATCH_ALIGN - 1) / BATCH_ALIGN * BATCH_ALIGN);
        }
        g.total = gz.back();
        if (int rc = cuda_ok(b, cudaMemcpy(g.items_dev, it.data(), it.size() * sizeof(BatchItem),
                                           cudaMemcpyHostToDevice), "upload group items"))
            return rc;
        if (int rc = cuda_ok(b, cudaMemcpy(g.zpad_dev, gz.data(), gz.size() * sizeof(long long),
                                           cudaMemcpyHostToDevice), "upload group offsets"))
            return rc;
    }
    return ADER_OK;
}

int launch_dt(ader_batch* b, double cfl, double* dt, cudaStream_t st) {
    BatchGroupDev g{b->all_items_dev, b->all_zpad_dev, b->n, b->all_total};
    const long long want = (b->all_total + 255) / 256;
    const int blocks = (int)std::min<long long>(want, (long long)b->sms * 8);
    kb_max_dt<<<blocks, 256, 0, st>>>(g, b->smax);
    kb_max_dt_finish<<<1, 256, 0, st>>>(b->n, cfl, b->smax, dt);
    return cuda_ok(b, cudaGetLastError(), "batched dt launch");
}

// Enqueues one step: [dt], fork, each group's phases on its stream, join.
int enqueue_step(ader_batch* b, bool with_dt, double cfl, double* dt, cudaStream_t st) {
    if (with_dt)
        if (int rc = launch_dt(b, cfl, dt, st)) return rc;
    if (int rc = cuda_ok(b, cudaEventRecord(b->fork, st), "fork record")) return rc;
    for (auto& g : b->groups) {
        if (int rc = cuda_ok(b, cudaStreamWaitEvent(g.stream, b->fork, 0), "fork wait")) return rc;
        for (int ph = 0; ph < PH_COUNT; ++ph) {
            if (!batch_phase_applies(ph, g.order, g.mhd)) continue;
            if (run_phase(g, ph, g.tuned[ph].threads, g.tuned[ph].blocks, g.stream, true, nullptr) < 0)
                return fail(b, ADER_ERR_CUDA, "batched phase launch");
        }
        if (int rc = cuda_ok(b, cudaEventRecord(g.done, g.stream), "join record")) return rc;
        if (int rc = cuda_ok(b, cudaStreamWaitEvent(st, g.done, 0), "join wait")) return rc;
    }
    return cuda_ok(b, cudaGetLastError(), "batched step launch");
}

bool valid_state(const ader_batch* b, double* const* U, double* const* Bf) {
    if (!U) return false;
    for (int p = 0; p < b->n; ++p) {
        if (!U[p]) return false;
        if (b->mhd[p] && (!Bf || !Bf[p])) return false;
    }
    return true;
}

int step_graph_on(ader_batch* b, double* const* U, double* const* Bf, bool with_dt, double cfl, double* dt_dev,
                  cudaStream_t st);

int step_graph(ader_batch* b, double* const* U, double* const* Bf, bool with_dt, double cfl, double* dt_dev,
               cudaStream_t st) {
    if (!valid_state(b, U, Bf)) return fail(b, ADER_ERR_ARG, "null state pointer (or face field of an MHD problem)");
    if (st) return step_graph_on(b, U, Bf, with_dt, cfl, dt_dev, st);
    if (int rc = cuda_ok(b, cudaEventRecord(b->bridge_in, st), "bridge record")) return rc;
    if (int rc = cuda_ok(b, cudaStreamWaitEvent(b->own, b->bridge_in, 0), "bridge wait")) return rc;
    if (int rc = step_graph_on(b, U, Bf, with_dt, cfl, dt_dev, b->own)) return rc;
    if (int rc = cuda_ok(b, cudaEventRecord(b->bridge_out, b->own), "bridge record")) return rc;
    return cuda_ok(b, cudaStreamWaitEvent(st, b->bridge_out, 0), "bridge wait");
}

int step_graph_on(ader_batch* b, double* const* U, double* const* Bf, bool with_dt, double cfl, double* dt_dev,
                  cudaStream_t st) {
    std::vector<const void*> key;
    key.push_back((const void*)(size_t)(with_dt ? 1 : 0));
    key.push_back(dt_dev);
    for (int p = 0; p < b->n; ++p) {
        key.push_back(U[p]);
        key.push_back(b->mhd[p] ? Bf[p] : nullptr);
    }
    if (!b->exec || key != b->key || (with_dt && cfl != b->key_cfl)) {
        // the tables are rewritten: let steps in flight that read them finish first
        if (int rc = cuda_ok(b, cudaStreamSynchronize(st), "sync before re-capture")) return rc;
        if (b->exec) {
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
        if (int rc = upload(b, U, Bf, dt_dev)) return rc;
        cudaGraph_t graph = nullptr;
        if (int rc = cuda_ok(b, cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "begin capture"))
            return rc;
        const int rc = enqueue_step(b, with_dt, cfl, dt_dev, st);
        const cudaError_t e = cudaStreamEndCapture(st, &graph);
        if (rc) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (int r2 = cuda_ok(b, e, "end capture")) return r2;
        const cudaError_t ei = cudaGraphInstantiate(&b->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (int r3 = cuda_ok(b, ei, "graph instantiate")) return r3;
        b->key = key;
        b->key_cfl = cfl;
    }
    return cuda_ok(b, cudaGraphLaunch(b->exec, st), "graph launch");
}

}  // namespace

extern "C" {

int ader_batch_create(int n, const ader_grid* grids, const int* orders, const double* gammas, const int* solvers,
                      const unsigned* flags, ader_batch** out) {
    if (!out) return ADER_ERR_ARG;
    *out = nullptr;
    if (n < 1 || n > ADER_BATCH_MAX || !grids || !orders || !gammas || !solvers || !flags) return ADER_ERR_ARG;
    const unsigned known = ADER_MHD | ADER_NODAL | ADER_FP32_BULK;
    for (int p = 0; p < n; ++p) {
        const ader_grid& g = grids[p];
        if (g.nx < 1 || g.ny < 1 || g.nz < 1 || !(g.dx > 0) || !(g.dy > 0) || !(g.dz > 0)) return ADER_ERR_ARG;
        if (orders[p] < 2 || orders[p] > 4 || !(gammas[p] > 1.0)) return ADER_ERR_ARG;
        if (solvers[p] != ADER_HLL && solvers[p] != ADER_LINEARIZED) return ADER_ERR_ARG;
        if ((flags[p] & ~known) || !(flags[p] & ADER_FP32_BULK)) return ADER_ERR_ARG;   // FP32 bulk only
    }
    ader_batch* b = new ader_batch();
    b->n = n;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    size_t bytes = 0;
    std::vector<size_t> off(n);
    auto align = [](size_t x) { return (x + 255) / 256 * 256; };
    for (int p = 0; p < n; ++p) {
        b->grids.push_back(grids[p]);
        b->order.push_back(orders[p]);
        b->solver.push_back(solvers[p]);
        b->mhd.push_back((flags[p] & ADER_MHD) ? 1 : 0);
        b->form.push_back((flags[p] & ADER_NODAL) ? FORM_NODAL : FORM_MODAL);
        b->gamma.push_back(gammas[p]);
        const long long N = (long long)grids[p].nx * grids[p].ny * grids[p].nz;
        b->zones.push_back(N);
        off[p] = bytes;
        const int m = b->mhd[p];
        const size_t per = (size_t)(s1_per_zone(orders[p], m) + std::max(1, s2_per_zone(orders[p], m)) +
                                    s3_per_zone(m, solvers[p] == ADER_LINEARIZED)) + (m ? 6 : 0) + 5;
        bytes += align(per * (size_t)N * sizeof(float) + 8 * 256);      // six arrays, each 256-B aligned
    }
    bool ok = cudaMalloc(&b->arena, bytes) == cudaSuccess;
    ok = ok && cudaMalloc((void**)&b->flags, n * sizeof(unsigned)) == cudaSuccess;
    ok = ok && cudaMalloc((void**)&b->dt_int, n * sizeof(double)) == cudaSuccess;
    ok = ok && cudaMalloc((void**)&b->smax, n * sizeof(unsigned long long)) == cudaSuccess;
    ok = ok && cudaMalloc((void**)&b->all_items_dev, n * sizeof(BatchItem)) == cudaSuccess;
    ok = ok && cudaMalloc((void**)&b->all_zpad_dev, (n + 1) * sizeof(long long)) == cudaSuccess;
    ok = ok && cudaMemset(b->flags, 0, n * sizeof(unsigned)) == cudaSuccess;
    ok = ok && cudaMemset(b->dt_int, 0, n * sizeof(double)) == cudaSuccess;
    ok = ok && cudaMemset(b->smax, 0, n * sizeof(unsigned long long)) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&b->bridge_in, cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&b->bridge_out, cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaStreamCreateWithFlags(&b->own, cudaStreamNonBlocking) == cudaSuccess;
    // per-problem step arguments
    for (int p = 0; p < n && ok; ++p) {
        BatchItem it;
        std::memset(&it, 0, sizeof(it));
        StepArgs& a = it.a;
        const long long N = b->zones[p];
        const int m = b->mhd[p];
        a.grid = Grid{grids[p].nx, grids[p].ny, grids[p].nz, N};
        a.order = orders[p];
        a.form = b->form[p];
        a.solver = solvers[p];
        a.fp32 = 1;
        a.n_iter = orders[p] - 1;
        a.tol = 0.0;
        a.max_iter = 50;
        a.gamma = gammas[p];
        a.dx[0] = grids[p].dx;
        a.dx[1] = grids[p].dy;
        a.dx[2] = grids[p].dz;
        finish_args(a);
        a.mhd = m;
        a.flag = b->flags + p;
        char* base = (char*)b->arena + off[p];
        auto take = [&](size_t count) {
            void* q = base;
            base += align(count * sizeof(float));
            return q;
        };
        a.S1 = take((size_t)s1_per_zone(orders[p], m) * N);
        a.S2 = take((size_t)std::max(1, s2_per_zone(orders[p], m)) * N);
        a.S3 = take((size_t)s3_per_zone(m, solvers[p] == ADER_LINEARIZED) * N);
        a.ZB = m ? take((size_t)3 * N) : nullptr;
        a.E = m ? take((size_t)3 * N) : nullptr;
        a.Uf = (const float*)take((size_t)5 * N);
        b->items.push_back(it);
    }
    // variant groups
    for (int p = 0; p < n && ok; ++p) {
        auto it = std::find_if(b->groups.begin(), b->groups.end(), [&](const Group& g) {
            return g.order == b->order[p] && g.mhd == b->mhd[p] && g.form == b->form[p] && g.solver == b->solver[p];
        });
        if (it == b->groups.end()) {
            Group g;
            g.order = b->order[p];
            g.mhd = b->mhd[p];
            g.form = b->form[p];
            g.solver = b->solver[p];
            b->groups.push_back(g);
            it = b->groups.end() - 1;
        }
        it->members.push_back(p);
    }
    for (auto& g : b->groups) {
        if (!ok) break;
        ok = ok && cudaMalloc((void**)&g.items_dev, g.members.size() * sizeof(BatchItem)) == cudaSuccess;
        ok = ok && cudaMalloc((void**)&g.zpad_dev, (g.members.size() + 1) * sizeof(long long)) == cudaSuccess;
        ok = ok && cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking) == cudaSuccess;
        ok = ok && cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming) == cudaSuccess;
    }
    if (!ok) {
        ader_batch_destroy(b);
        return ADER_ERR_CUDA;
    }
    *out = b;
    return ADER_OK;
}

int ader_batch_step(ader_batch* b, double* const* U, double* const* Bface, const double* dt_dev, void* stream) {
    if (!b) return ADER_ERR_ARG;
    if (!dt_dev) return fail(b, ADER_ERR_ARG, "dt_dev is null");
    return step_graph(b, U, Bface, false, 0.0, const_cast<double*>(dt_dev), (cudaStream_t)stream);
}

int ader_batch_advance(ader_batch* b, double* const* U, double* const* Bface, double cfl, double* dt_dev,
                       void* stream) {
    if (!b) return ADER_ERR_ARG;
    if (!(cfl > 0.0)) return fail(b, ADER_ERR_ARG, "cfl must be positive");
    return step_graph(b, U, Bface, true, cfl, dt_dev ? dt_dev : b->dt_int, (cudaStream_t)stream);
}

int ader_batch_tune(ader_batch* b, double* const* U, double* const* Bface, void* stream) {
    if (!b) return ADER_ERR_ARG;
    if (!valid_state(b, U, Bface)) return fail(b, ADER_ERR_ARG, "null state pointer");
    cudaStream_t st = (cudaStream_t)stream;
    if (int rc = cuda_ok(b, cudaStreamSynchronize(st), "sync before tuning")) return rc;
    if (int rc = cuda_ok(b, cudaStreamSynchronize(b->own), "sync before tuning")) return rc;
    // private copies: the update phases write the state in place
    std::vector<double*> Uc(b->n, nullptr), Bc(b->n, nullptr);
    int rc = ADER_OK;
    for (int p = 0; p < b->n && rc == ADER_OK; ++p) {
        const size_t nz = (size_t)b->zones[p];
        rc = cuda_ok(b, cudaMalloc((void**)&Uc[p], 5 * nz * sizeof(double)), "tune copy");
        if (rc == ADER_OK) rc = cuda_ok(b, cudaMemcpyAsync(Uc[p], U[p], 5 * nz * sizeof(double),
                                                           cudaMemcpyDeviceToDevice, st), "tune copy");
        if (rc == ADER_OK && b->mhd[p]) {
            rc = cuda_ok(b, cudaMalloc((void**)&Bc[p], 3 * nz * sizeof(double)), "tune copy");
            if (rc == ADER_OK) rc = cuda_ok(b, cudaMemcpyAsync(Bc[p], Bface[p], 3 * nz * sizeof(double),
                                                               cudaMemcpyDeviceToDevice, st), "tune copy");
        }
    }
    if (rc == ADER_OK) rc = upload(b, Uc.data(), Bc.data(), nullptr);
    if (rc == ADER_OK) rc = launch_dt(b, 0.2, b->dt_int, st);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (rc == ADER_OK) rc = cuda_ok(b, cudaEventCreate(&e0), "event");
    if (rc == ADER_OK) rc = cuda_ok(b, cudaEventCreate(&e1), "event");
    const int Ts[3] = {64, 128, 256};
    for (auto& g : b->groups) {
        for (int ph = 0; ph < PH_COUNT && rc == ADER_OK; ++ph) {
            if (!batch_phase_applies(ph, g.order, g.mhd)) continue;
            Tuned best;
            for (int T : Ts) {
                if (T > batch_phase_max_threads(ph)) continue;
                const void* fn = nullptr;
                run_phase(g, ph, T, 1, st, false, &fn);
                int occ = 0;
                if (!fn || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, T, 0) != cudaSuccess || occ < 1)
                    continue;
                const long long full = (g.total + T - 1) / T;
                const int cand[5] = {b->sms * occ, b->sms * occ * 2, b->sms * occ * 4, b->sms * occ * 8, 0};
                for (int B : cand) {
                    if (B > 0 && (B >= full || !batch_phase_persistent(ph))) continue;   // same as the full grid
                    // one warm-up, then the best of three
                    if (run_phase(g, ph, T, B, st, true, nullptr) < 0) {
                        rc = fail(b, ADER_ERR_CUDA, "tuning launch");
                        break;
                    }
                    float bestms = 1e30f;
                    for (int r = 0; r < 3 && rc == ADER_OK; ++r) {
                        cudaEventRecord(e0, st);
                        run_phase(g, ph, T, B, st, true, nullptr);
                        cudaEventRecord(e1, st);
                        rc = cuda_ok(b, cudaEventSynchronize(e1), "tuning sync");
                        float ms = 0.f;
                        cudaEventElapsedTime(&ms, e0, e1);
                        bestms = std::min(bestms, ms);
                    }
                    if (rc != ADER_OK) break;
                    if (best.ms < 0.f || bestms < best.ms) {
                        best.threads = T;
                        best.blocks = B;
                        best.ms = bestms;
                    }
                }
                if (rc != ADER_OK) break;
            }
            if (best.ms >= 0.f) g.tuned[ph] = best;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(st);
    for (int p = 0; p < b->n; ++p) {
        if (Uc[p]) cudaFree(Uc[p]);
        if (Bc[p]) cudaFree(Bc[p]);
    }
    cudaMemsetAsync(b->flags, 0, b->n * sizeof(unsigned), st);   // flags raised on the copies do not count
    cudaStreamSynchronize(st);
    if (b->exec) {                                                 // the captured graph used the old shapes
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
        b->key.clear();
    }
    b->tuned = rc == ADER_OK;
    return rc;
}

int ader_batch_tuning(const ader_batch* b, int* out_host, int cap) {
    if (!b || !out_host) return ADER_ERR_ARG;
    int k = 0;
    for (size_t gi = 0; gi < b->groups.size(); ++gi) {
        const Group& g = b->groups[gi];
        for (int ph = 0; ph < PH_COUNT; ++ph) {
            if (!batch_phase_applies(ph, g.order, g.mhd)) continue;
            if (k + 4 <= cap) {
                out_host[k] = (int)gi;
                out_host[k + 1] = ph;
                out_host[k + 2] = g.tuned[ph].threads;
                out_host[k + 3] = g.tuned[ph].blocks;
            }
            k += 4;
        }
    }
    return k / 4;
}

int ader_batch_status(ader_batch* b, int* codes_host, void* stream) {
    if (!b) return ADER_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<unsigned> h(b->n, 0);
    int rc = cuda_ok(b, cudaMemcpyAsync(h.data(), b->flags, b->n * sizeof(unsigned), cudaMemcpyDeviceToHost, st),
                     "status read");
    if (rc == ADER_OK) rc = cuda_ok(b, cudaMemsetAsync(b->flags, 0, b->n * sizeof(unsigned), st), "status clear");
    if (rc == ADER_OK) rc = cuda_ok(b, cudaStreamSynchronize(st), "status sync");
    if (rc != ADER_OK) return rc;
    int worst = ADER_OK;
    for (int p = 0; p < b->n; ++p) {
        int c = ADER_OK;
        if (h[p] & FLAG_NONFINITE)
            c = ADER_ERR_NONFINITE;
        else if (h[p] & FLAG_UNPHYSICAL)
            c = ADER_ERR_UNPHYSICAL;
        if (codes_host) codes_host[p] = c;
        if (c != ADER_OK && worst == ADER_OK) worst = c;
    }
    if (worst != ADER_OK) b->err = "a problem of the batch reported a device error (see the per-problem codes)";
    return worst;
}

int ader_batch_groups(const ader_batch* b) { return b ? (int)b->groups.size() : 0; }

const char* ader_batch_last_error(const ader_batch* b) { return b ? b->err.c_str() : "null batch"; }

void ader_batch_destroy(ader_batch* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (auto& g : b->groups) {
        if (g.items_dev) cudaFree(g.items_dev);
        if (g.zpad_dev) cudaFree(g.zpad_dev);
        if (g.stream) cudaStreamDestroy(g.stream);
        if (g.done) cudaEventDestroy(g.done);
    }
    void* ptrs[] = {b->arena, b->flags, b->dt_int, b->smax, b->all_items_dev, b->all_zpad_dev};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->bridge_in) cudaEventDestroy(b->bridge_in);
    if (b->bridge_out) cudaEventDestroy(b->bridge_out);
    if (b->own) cudaStreamDestroy(b->own);
    delete b;
}

}  // extern "C"
