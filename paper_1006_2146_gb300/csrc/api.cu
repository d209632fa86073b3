// C ABI of the library (include/ader.h): context, scratch ownership, step
// sequencing and error reporting.  Every numerical step runs in the kernels
// of recon.cu, step_o*.cu and reduce.cu.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/ader.h"
#include "kernels.cuh"

using namespace ader;

struct ader_ctx {
    ader_grid g;
    Grid grid;
    int order, solver;
    unsigned flags;
    double gamma;
    bool fp32;
    size_t rsize;                 // bytes per bulk scalar (4 or 8)
    void* S1 = nullptr;
    void* S2 = nullptr;
    void* S3 = nullptr;
    void* ZB = nullptr;                       // MHD: zone field from the face-B WENO
    void* E = nullptr;                        // MHD: edge EMFs
    bool mhd = false;
    unsigned* flag = nullptr;                 // device error flag
    unsigned long long* dtscr = nullptr;      // max_dt scratch (2 words)
    double* partial = nullptr;                // totals partials
    int tot_blocks = 0;
    double* dt_dev = nullptr;                 // device dt of the host-memory path
    double* Ustage = nullptr;                 // device state of the host-memory path
    double* rk[7] = {};                       // SSP-RK stage states and operators
    double* rkB[6] = {};                      // MHD: SSP-RK stage face fields and the stored operator
    double tol = 0.0;                         // converged predictor tolerance (0: fixed M-1 iterations)
    int max_iter = 50;
    bool tiled = true;                        // Euler: per-tile predictor and face solves (ader_set_tiled)
    bool wait_test = false;                   // the next learned-guess launch tests its bounded waits
    int bc[6] = {0, 0, 0, 0, 0, 0};           // box faces (ader_set_boundary); all periodic by default
    int ghosts[3] = {0, 0, 0};                // ghost zones per side of each non-periodic axis
    ader_ctx* inner = nullptr;                // non-periodic faces: the context of the padded grid
    double* Upad = nullptr;                   // the padded state (5 x padded zones FP64)
    unsigned long long* stats = nullptr;      // converged predictor statistics (3 words)
    const float* guess = nullptr;             // learned-guess MLP parameters (device), order 3
    float* G = nullptr;                       // per-zone learned guess (5 x NV x N FP32), allocated by ader_set_guess
    int* Glist = nullptr;                     // the zones with slopes (N), their count and per-zone flags,
    unsigned* Gcount = nullptr;               // allocated with G
    unsigned char* Gact = nullptr;
    float* Uf = nullptr;                      // FP32 bulk: the state rounded to FP32 (5 x N), rewritten each step
    int src_kind = SOURCE_NONE;               // non-stiff source (ader_set_source)
    double src_par[3] = {0.0, 0.0, 0.0};
    void* Sb = nullptr;                       // dt S-bar per zone (5 x N, bulk precision), allocated with the source
    void* Dm = nullptr;                       // dense output: the last step's space-time modes (L x NV x N, bulk)
    double* Uold = nullptr;                   // positivity fallback: U^n of the current step (5 x N FP64)
    double* Bold = nullptr;                   // MHD positivity fallback: the face field of step n (3 x N FP64)
    unsigned char* pmark = nullptr;           // positivity fallback: zones marked non-physical (N bytes)
    bool dense_valid = false;                 // a step has written Dm since it was allocated
    bool setup_failed = false;                // a kernel could not be configured while enqueuing
    int launches = 0;
    std::string err;
    // tracing: pending event pairs per kernel name, folded into totals on read
    bool profiling = false;
    struct Pending { const char* name; cudaEvent_t a, b; };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> spare;
    std::vector<const char*> tnames;
    std::vector<int> tcount;
    std::vector<double> tms;
};

// Brackets one kernel launch with events when tracing is on.
struct Trace {
    ader_ctx* c;
    const char* name;
    cudaStream_t st;
    cudaEvent_t a = nullptr, b = nullptr;
    static cudaEvent_t take(ader_ctx* c) {
        if (!c->spare.empty()) {
            cudaEvent_t e = c->spare.back();
            c->spare.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    Trace(ader_ctx* c_, const char* n, cudaStream_t s) : c(c_), name(n), st(s) {
        if (c && c->profiling) {
            a = take(c);
            b = take(c);
            cudaEventRecord(a, st);
        }
    }
    ~Trace() {
        if (a) {
            cudaEventRecord(b, st);
            c->pending.push_back({name, a, b});
        }
    }
};

static int fail(ader_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    return code;
}

static int cuda_check(ader_ctx* c, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return ADER_OK;
    return fail(c, ADER_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

static StepArgs make_args(const ader_ctx* c, double dt, const double* dt_dev, int n_iter) {
    StepArgs a;
    a.grid = c->grid;
    a.order = c->order;
    a.form = (c->flags & ADER_NODAL) ? FORM_NODAL : FORM_MODAL;
    a.solver = c->solver;
    a.fp32 = c->fp32 ? 1 : 0;
    a.n_iter = n_iter;
    a.gamma = c->gamma;
    a.dx[0] = c->g.dx;
    a.dx[1] = c->g.dy;
    a.dx[2] = c->g.dz;
    finish_args(a);
    a.Uf = c->Uf;
    a.dt = dt;
    a.dt_dev = dt_dev;
    a.S1 = c->S1;
    a.S2 = c->S2;
    a.S3 = c->S3;
    a.flag = c->flag;
    a.mhd = c->mhd ? 1 : 0;
    a.Bface = nullptr;
    a.ZB = c->ZB;
    a.E = c->E;
    a.tol = n_iter > 0 ? c->tol : 0.0;
    a.max_iter = c->max_iter;
    a.stats = c->stats;
    a.guess = n_iter > 0 ? c->guess : nullptr;
    a.G = a.guess ? c->G : nullptr;
    a.Glist = c->Glist;
    a.Gcount = c->Gcount;
    a.Gact = a.G ? c->Gact : nullptr;
    a.src_kind = n_iter > 0 ? c->src_kind : SOURCE_NONE;
    for (int i = 0; i < 3; ++i) a.src_par[i] = c->src_par[i];
    a.Sb = a.src_kind != SOURCE_NONE ? c->Sb : nullptr;
    a.modes_out = nullptr;
    a.emf_transonic = (c->flags & ADER_EMF_TRANSONIC) ? 1 : 0;
    a.defer_nonfinite = 0;
    a.tiled = c->tiled ? 1 : 0;               // the predictor tiles check the physics and order themselves
    a.wait_test = c->wait_test ? 1 : 0;
    return a;
}

template <class R>
static int enqueue_faces(ader_ctx* c, const StepArgs& a, const double* U, cudaStream_t st) {
    int n;
    {
        Trace t(c, "weno_reconstruction", st);
        n = launch_recon<R>(a, U, st);
    }
    if (a.G) {
        Trace t(c, "learned_guess", st);
        c->wait_test = false;                 // one launch only
        const int k = launch_guess<R>(a, U, st, nullptr);
        if (k < 0)
            c->setup_failed = true;       // reported by the caller
        else
            n += k;
    }
    Trace t(c, "predictor_faces", st);
    if (a.mhd) {
        switch (a.order) {
            case 2: n += launch_predict_faces_nv<2, 8, R>(a, U, st); break;
            case 3: n += launch_predict_faces_nv<3, 8, R>(a, U, st); break;
            default: n += launch_predict_faces_nv<4, 8, R>(a, U, st); break;
        }
    } else {
        switch (a.order) {
            case 2: n += launch_predict_faces_nv<2, 5, R>(a, U, st); break;
            case 3: n += launch_predict_faces_nv<3, 5, R>(a, U, st); break;
            default: n += launch_predict_faces_nv<4, 5, R>(a, U, st); break;
        }
    }
    return n;
}

// out = base + c * L(U) after computing the face data of U
static int enqueue_operator(ader_ctx* c, const StepArgs& a, const double* U, double* out, const double* base,
                            double coef, bool use_dt_dev, cudaStream_t st) {
    int n = c->fp32 ? enqueue_faces<float>(c, a, U, st) : enqueue_faces<double>(c, a, U, st);
    Trace t(c, "riemann_update", st);
    n += c->fp32 ? launch_flux_update<float>(a, out, base, coef, use_dt_dev, st)
                 : launch_flux_update<double>(a, out, base, coef, use_dt_dev, st);
    return n;
}

extern "C" {

int ader_create(const ader_grid* g, int order, double gamma, int solver, unsigned flags, ader_ctx** out) {
    if (!out) return ADER_ERR_ARG;
    *out = nullptr;
    if (!g || g->nx < 1 || g->ny < 1 || g->nz < 1 || !(g->dx > 0) || !(g->dy > 0) || !(g->dz > 0))
        return ADER_ERR_ARG;
    if (order < 2 || order > 4 || !(gamma > 1.0) || (solver != ADER_HLL && solver != ADER_LINEARIZED))
        return ADER_ERR_ARG;
    const unsigned known = ADER_MHD | ADER_NODAL | ADER_FP32_BULK | ADER_EMF_TRANSONIC | ADER_POSITIVITY_FALLBACK;
    if ((flags & ADER_POSITIVITY_FALLBACK) && (flags & ADER_FP32_BULK)) return ADER_ERR_ARG;
    if (flags & ~known) return ADER_ERR_ARG;        // the converged predictor is set by ader_set_predictor
    ader_ctx* c = new ader_ctx();
    c->g = *g;
    c->grid.nx = g->nx;
    c->grid.ny = g->ny;
    c->grid.nz = g->nz;
    c->grid.n = (long long)g->nx * g->ny * g->nz;
    c->order = order;
    c->solver = solver;
    c->flags = flags;
    c->gamma = gamma;
    c->fp32 = (flags & ADER_FP32_BULK) != 0;
    c->rsize = c->fp32 ? 4 : 8;
    c->mhd = (flags & ADER_MHD) != 0;
    const int mh = c->mhd ? 1 : 0;
    const size_t N = (size_t)c->grid.n;
    int rc = ADER_OK;
    auto alloc = [&](void** p, size_t bytes, const char* what) {
        if (rc != ADER_OK || bytes == 0) return;
        rc = cuda_check(c, cudaMalloc(p, bytes), what);
    };
    alloc(&c->S1, N * s1_per_zone(order, mh) * c->rsize, "cudaMalloc S1");
    alloc(&c->S2, N * (s2_per_zone(order, mh) ? s2_per_zone(order, mh) : 1) * c->rsize, "cudaMalloc S2");
    alloc(&c->S3, N * s3_per_zone(mh, solver == ADER_LINEARIZED) * c->rsize, "cudaMalloc S3");
    if (c->mhd) {
        alloc(&c->ZB, N * 3 * c->rsize, "cudaMalloc zone B");
        alloc(&c->E, N * 3 * c->rsize, "cudaMalloc EMF");
    }
    if (c->fp32) alloc((void**)&c->Uf, N * 5 * sizeof(float), "cudaMalloc FP32 state copy");
    if (flags & ADER_POSITIVITY_FALLBACK) {
        alloc((void**)&c->Uold, N * 5 * sizeof(double), "cudaMalloc U^n copy");
        alloc((void**)&c->pmark, N, "cudaMalloc positivity marks");
        if (c->mhd) alloc((void**)&c->Bold, N * 3 * sizeof(double), "cudaMalloc B^n copy");
    }
    alloc((void**)&c->flag, sizeof(unsigned), "cudaMalloc flag");
    alloc((void**)&c->stats, 3 * sizeof(unsigned long long), "cudaMalloc predictor statistics");
    alloc((void**)&c->dtscr, 2 * sizeof(unsigned long long), "cudaMalloc dt scratch");
    c->tot_blocks = 1024;
    alloc((void**)&c->partial, c->tot_blocks * 10 * sizeof(double), "cudaMalloc partials");
    alloc((void**)&c->dt_dev, sizeof(double), "cudaMalloc dt");
    alloc((void**)&c->Ustage, N * 5 * sizeof(double), "cudaMalloc host-path state");
    for (int s = 0; s < 7; ++s) alloc((void**)&c->rk[s], N * 5 * sizeof(double), "cudaMalloc RK stage");
    if (c->mhd)
        for (int s = 0; s < 6; ++s) alloc((void**)&c->rkB[s], N * 3 * sizeof(double), "cudaMalloc RK face field");
    if (rc == ADER_OK) rc = cuda_check(c, cudaMemset(c->flag, 0, sizeof(unsigned)), "cudaMemset flag");
    if (rc == ADER_OK) rc = cuda_check(c, cudaMemset(c->stats, 0, 3 * sizeof(unsigned long long)), "cudaMemset");
    if (rc == ADER_OK) rc = cuda_check(c, cudaMemset(c->dtscr, 0, 2 * sizeof(unsigned long long)), "cudaMemset");
    if (rc != ADER_OK) {
        ader_destroy(c);
        return rc;
    }
    *out = c;
    return ADER_OK;
}

void ader_destroy(ader_ctx* c) {
    if (!c) return;
    if (c->inner) {              // it shares the flag and the predictor statistics of this context
        c->inner->flag = nullptr;
        c->inner->stats = nullptr;
        ader_destroy(c->inner);
        c->inner = nullptr;
    }
    if (c->Upad) cudaFree(c->Upad);
    for (auto& p : c->pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (auto e : c->spare) cudaEventDestroy(e);
    void* ptrs[] = {c->S1, c->S2, c->S3, c->ZB, c->E, c->G, c->Glist, c->Gact, c->Gcount, c->Uf, c->Sb, c->Dm, c->Uold, c->Bold, c->pmark, c->flag,
                    c->stats, c->dtscr, c->partial, c->dt_dev,
                    c->Ustage, c->rk[0], c->rk[1], c->rk[2], c->rk[3], c->rk[4], c->rk[5], c->rk[6],
                    c->rkB[0], c->rkB[1], c->rkB[2], c->rkB[3], c->rkB[4], c->rkB[5]};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete c;
}

const char* ader_last_error(const ader_ctx* c) { return c ? c->err.c_str() : "null context"; }

int ader_launches_per_step(const ader_ctx* c) { return c ? c->launches : 0; }

int ader_profile(ader_ctx* c, int enable) {
    if (!c) return ADER_ERR_ARG;
    c->profiling = enable != 0;
    return ADER_OK;
}

int ader_profile_reset(ader_ctx* c) {
    if (!c) return ADER_ERR_ARG;
    for (auto& p : c->pending) {
        c->spare.push_back(p.a);
        c->spare.push_back(p.b);
    }
    c->pending.clear();
    c->tnames.clear();
    c->tcount.clear();
    c->tms.clear();
    return ADER_OK;
}

int ader_profile_read(ader_ctx* c, const char** names, int* launches, double* ms, int cap) {
    if (!c) return ADER_ERR_ARG;
    for (auto& p : c->pending) {
        cudaError_t e = cudaEventSynchronize(p.b);
        if (e != cudaSuccess) return cuda_check(c, e, "cudaEventSynchronize");
        float t = 0.f;
        cudaEventElapsedTime(&t, p.a, p.b);
        size_t k = 0;
        while (k < c->tnames.size() && strcmp(c->tnames[k], p.name) != 0) ++k;
        if (k == c->tnames.size()) {
            c->tnames.push_back(p.name);
            c->tcount.push_back(0);
            c->tms.push_back(0.0);
        }
        c->tcount[k] += 1;
        c->tms[k] += t;
        c->spare.push_back(p.a);
        c->spare.push_back(p.b);
    }
    c->pending.clear();
    const int n = (int)c->tnames.size();
    for (int k = 0; k < n && k < cap; ++k) {
        if (names) names[k] = c->tnames[k];
        if (launches) launches[k] = c->tcount[k];
        if (ms) ms[k] = c->tms[k];
    }
    return n;
}

static int check_bface(ader_ctx* c, const double* Bface) {
    if (c->mhd && !Bface) return fail(c, ADER_ERR_ARG, "MHD context: Bface is required");
    if (!c->mhd && Bface) return fail(c, ADER_ERR_ARG, "Euler context: Bface must be null");
    return ADER_OK;
}

static int step_common(ader_ctx* c, double* U, double* Bface, double dt, const double* dt_dev, void* stream);

// Non-periodic faces: fill the padded state's ghost zones from U, step it with the padded grid's
// context, copy its interior back to U.
static int step_padded(ader_ctx* c, double* U, double dt, const double* dt_dev, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    ader_ctx* in = c->inner;
    {
        Trace t(c, "boundary_ghosts", st);
        launch_fill_ghosts(c->grid, in->grid, c->bc, c->ghosts, U, c->Upad, st);
    }
    if (int rc = step_common(in, c->Upad, nullptr, dt, dt_dev, stream)) return fail(c, rc, in->err);
    {
        Trace t(c, "boundary_interior", st);
        launch_copy_interior(c->grid, in->grid, c->ghosts, c->Upad, U, st);
    }
    c->launches = in->launches + 2;
    return cuda_check(c, cudaGetLastError(), "ader_step launch");
}

static int step_common(ader_ctx* c, double* U, double* Bface, double dt, const double* dt_dev, void* stream) {
    if (!c) return ADER_ERR_ARG;
    if (!U) return fail(c, ADER_ERR_ARG, "U is null");
    if (int rc = check_bface(c, Bface)) return rc;
    if (!dt_dev && !(dt > 0.0)) return fail(c, ADER_ERR_ARG, "dt must be positive");
    if (c->inner) return step_padded(c, U, dt, dt_dev, stream);
    cudaStream_t st = (cudaStream_t)stream;
    StepArgs a = make_args(c, dt, dt_dev, c->order - 1);
    a.Bface = Bface;
    a.modes_out = c->Dm;
    a.defer_nonfinite = c->Uold ? 1 : 0;     // the fallback mends non-finite zones, then checks them
    const double coef = dt_dev ? 1.0 : dt;
    if (c->Uold)
        if (int rc = cuda_check(c, cudaMemcpyAsync(c->Uold, U, (size_t)c->grid.n * 5 * sizeof(double),
                                                   cudaMemcpyDeviceToDevice, st), "copy of U^n"))
            return rc;
    if (c->Bold)
        if (int rc = cuda_check(c, cudaMemcpyAsync(c->Bold, Bface, (size_t)c->grid.n * 3 * sizeof(double),
                                                   cudaMemcpyDeviceToDevice, st), "copy of B^n"))
            return rc;
    c->launches = enqueue_operator(c, a, U, U, U, coef, dt_dev != nullptr, st);
    if (c->Dm) c->dense_valid = true;
    if (c->setup_failed) {
        c->setup_failed = false;
        return fail(c, ADER_ERR_CUDA, "learned-guess kernel set-up failed");
    }
    if (c->mhd) {
        Trace t(c, "emf_ct", st);
        c->launches += c->fp32 ? launch_emf_ct<float>(a, Bface, coef, dt_dev != nullptr, st)
                               : launch_emf_ct<double>(a, Bface, coef, dt_dev != nullptr, st);
    }
    if (c->Uold) {          // after constrained transport: an MHD zone's pressure takes the new face field
        Trace t(c, "positivity_fallback", st);
        c->launches += launch_positivity_fallback(a, U, c->Uold, c->Bold, c->pmark, coef, dt_dev != nullptr, st);
    }
    return cuda_check(c, cudaGetLastError(), "ader_step launch");
}

int ader_step(ader_ctx* c, double* U, double* Bface, double dt, void* stream) {
    return step_common(c, U, Bface, dt, nullptr, stream);
}

int ader_step_devdt(ader_ctx* c, double* U, double* Bface, const double* dt_dev, void* stream) {
    if (c && !dt_dev) return fail(c, ADER_ERR_ARG, "dt_dev is null");
    return step_common(c, U, Bface, 0.0, dt_dev, stream);
}

int ader_max_dt(ader_ctx* c, const double* U, const double* Bface, double cfl, double* dt_dev, void* stream) {
    if (!c) return ADER_ERR_ARG;
    if (!U || !dt_dev) return fail(c, ADER_ERR_ARG, "null pointer");
    if (int rc = check_bface(c, Bface)) return rc;
    if (!(cfl > 0.0)) return fail(c, ADER_ERR_ARG, "cfl must be positive");
    const double dx[3] = {c->g.dx, c->g.dy, c->g.dz};
    Trace t(c, "max_dt", (cudaStream_t)stream);
    launch_max_dt(c->grid, U, Bface, c->gamma, dx, cfl, dt_dev, c->dtscr, c->flag, c->fp32, (cudaStream_t)stream);
    return cuda_check(c, cudaGetLastError(), "ader_max_dt launch");
}

int ader_diagnostics(ader_ctx* c, const double* U, const double* Bface, double* totals_dev, void* stream) {
    if (!c) return ADER_ERR_ARG;
    if (!U || !totals_dev) return fail(c, ADER_ERR_ARG, "null pointer");
    if (int rc = check_bface(c, Bface)) return rc;
    const double dx[3] = {c->g.dx, c->g.dy, c->g.dz};
    launch_totals(c->grid, U, c->mhd ? Bface : nullptr, dx, totals_dev, c->partial, c->tot_blocks,
                  (cudaStream_t)stream);
    return cuda_check(c, cudaGetLastError(), "ader_diagnostics launch");
}

// SSP-RK stage tables of Eqs. 18-20: U(s) = sum_j A[s][j] U(j) + dt sum_j B[s][j] L(U(j))
static const double RK2A[2][2] = {{1.0, 0.0}, {0.5, 0.5}};
static const double RK2B[2][2] = {{1.0, 0.0}, {0.0, 0.5}};
static const double RK3A[3][3] = {{1.0, 0, 0}, {0.75, 0.25, 0}, {1.0 / 3.0, 0.0, 2.0 / 3.0}};
static const double RK3B[3][3] = {{1.0, 0, 0}, {0.0, 0.25, 0}, {0.0, 0.0, 2.0 / 3.0}};
static const double RK4A[5][5] = {{1.0, 0, 0, 0, 0},
                                  {0.44437049406734, 0.55562950593266, 0, 0, 0},
                                  {0.62010185138540, 0.0, 0.37989814861460, 0, 0},
                                  {0.17807995410773, 0.0, 0.0, 0.82192004589227, 0},
                                  {0.00683325884039, 0.0, 0.51723167208978, 0.12759831133288, 0.34833675773694}};
static const double RK4B[5][5] = {{0.39175222700392, 0, 0, 0, 0},
                                  {0.0, 0.36841059262959, 0, 0, 0},
                                  {0.0, 0.0, 0.25189177424738, 0, 0},
                                  {0.0, 0.0, 0.0, 0.54497475021237, 0},
                                  {0.0, 0.0, 0.0, 0.08460416338212, 0.22600748319395}};

int ader_rk_step(ader_ctx* c, double* U, double* Bface, double dt, void* stream) {
    if (!c) return ADER_ERR_ARG;
    if (!U) return fail(c, ADER_ERR_ARG, "U is null");
    if (int rc = check_bface(c, Bface)) return rc;
    if (!(dt > 0.0)) return fail(c, ADER_ERR_ARG, "dt must be positive");
    if (c->src_kind != SOURCE_NONE) return fail(c, ADER_ERR_ARG, "SSP-RK with a source term is not built");
    if (c->inner) return fail(c, ADER_ERR_ARG, "SSP-RK with non-periodic faces is not built");
    cudaStream_t st = (cudaStream_t)stream;
    const bool mhd = c->mhd;
    const int ns = c->order == 2 ? 2 : (c->order == 3 ? 3 : 5);
    const double* A = c->order == 2 ? &RK2A[0][0] : (c->order == 3 ? &RK3A[0][0] : &RK4A[0][0]);
    const double* B = c->order == 2 ? &RK2B[0][0] : (c->order == 3 ? &RK3B[0][0] : &RK4B[0][0]);
    const StepArgs a0 = make_args(c, dt, nullptr, 0);
    const long long cnt = c->grid.n * 5, cntB = c->grid.n * 3;
    // states[0] = U^n (copied), states[s] = U(s); ops[s] = L(U(s)) (stored only where reused);
    // for MHD the same for the face field (its operator is -curl E, the rate of Eq. 8)
    double* states[5] = {c->rk[0], c->rk[1], c->rk[2], c->rk[3], c->rk[4]};
    double* ops[2] = {c->rk[5], c->rk[6]};
    double* statesB[5] = {c->rkB[0], c->rkB[1], c->rkB[2], c->rkB[3], c->rkB[4]};
    double* opsB = c->rkB[5];
    int n = 0;
    cudaError_t e = cudaMemcpyAsync(states[0], U, cnt * sizeof(double), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && mhd)
        e = cudaMemcpyAsync(statesB[0], Bface, cntB * sizeof(double), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_check(c, e, "cudaMemcpyAsync");
    for (int s = 0; s < ns; ++s) {
        const double* rowA = A + s * ns;
        const double* rowB = B + s * ns;
        StepArgs a = a0;
        a.Bface = mhd ? statesB[s] : nullptr;          // the stage's face field (face-B WENO, EMFs)
        // state part of the stage
        const double* X[6];
        const double* XB[6];
        double w[6];
        int m = 0;
        for (int j = 0; j <= s; ++j)
            if (rowA[j] != 0.0) {
                X[m] = states[j];
                XB[m] = mhd ? statesB[j] : nullptr;
                w[m++] = rowA[j];
            }
        // operator terms other than L(U(s)) come from stored operators (only SSP(5,4)'s last stage)
        if (ns == 5 && s == 4) {
            X[m] = ops[0];          // L(U(3)) stored at stage 3
            XB[m] = opsB;
            w[m++] = rowB[3] * dt;
        }
        double* dst = (s == ns - 1) ? U : states[s + 1];
        double* dstB = mhd ? ((s == ns - 1) ? Bface : statesB[s + 1]) : nullptr;
        {
            Trace t(c, "rk_combine", st);
            n += launch_lincomb(dst, m, X, w, cnt, st);
            if (mhd) n += launch_lincomb(dstB, m, XB, w, cntB, st);
        }
        if (ns == 5 && s == 3) {
            // keep L(U(3)) (and L(B(3))) for the final stage, then dst += B[3][3] dt L(U(3))
            n += enqueue_operator(c, a, states[3], ops[0], nullptr, 1.0, false, st);
            if (mhd) {
                if (int rc = cuda_check(c, cudaMemsetAsync(opsB, 0, cntB * sizeof(double), st), "cudaMemsetAsync"))
                    return rc;
                Trace t(c, "emf_ct", st);
                n += c->fp32 ? launch_emf_ct<float>(a, opsB, 1.0, false, st) : launch_emf_ct<double>(a, opsB, 1.0, false, st);
            }
            const double* Y[2] = {dst, ops[0]};
            const double wy[2] = {1.0, rowB[3] * dt};
            Trace t(c, "rk_combine", st);
            n += launch_lincomb(dst, 2, Y, wy, cnt, st);
            if (mhd) {
                const double* YB[2] = {dstB, opsB};
                n += launch_lincomb(dstB, 2, YB, wy, cntB, st);
            }
        } else {
            n += enqueue_operator(c, a, states[s], dst, dst, rowB[s] * dt, false, st);
            if (mhd) {
                Trace t(c, "emf_ct", st);
                n += c->fp32 ? launch_emf_ct<float>(a, dstB, rowB[s] * dt, false, st)
                             : launch_emf_ct<double>(a, dstB, rowB[s] * dt, false, st);
            }
        }
    }
    c->launches = n + 1;
    return cuda_check(c, cudaGetLastError(), "ader_rk_step launch");
}

int ader_set_tiled(ader_ctx* c, int on) {
    if (!c) return ADER_ERR_ARG;
    c->tiled = on != 0;
    if (c->inner) c->inner->tiled = c->tiled;
    return ADER_OK;
}

int ader_set_boundary(ader_ctx* c, const int* bc) {
    if (!c) return ADER_ERR_ARG;
    if (!bc) return fail(c, ADER_ERR_ARG, "bc is null");
    bool any = false;
    for (int s = 0; s < 6; ++s) {
        if (bc[s] != ADER_BC_PERIODIC && bc[s] != ADER_BC_OUTFLOW && bc[s] != ADER_BC_REFLECTIVE)
            return fail(c, ADER_ERR_ARG, "unknown boundary code");
        any |= bc[s] != ADER_BC_PERIODIC;
    }
    const int n[3] = {c->grid.nx, c->grid.ny, c->grid.nz};
    const int G = c->order == 4 ? 4 : 3;       // a step's reach along an axis
    int gh[3];
    for (int d = 0; d < 3; ++d) {
        if ((bc[2 * d] == ADER_BC_PERIODIC) != (bc[2 * d + 1] == ADER_BC_PERIODIC))
            return fail(c, ADER_ERR_ARG, "an axis is periodic on both faces or on neither");
        gh[d] = bc[2 * d] == ADER_BC_PERIODIC ? 0 : G;
        if ((bc[2 * d] == ADER_BC_REFLECTIVE || bc[2 * d + 1] == ADER_BC_REFLECTIVE) && n[d] < G)
            return fail(c, ADER_ERR_ARG, "a reflecting face needs at least the ghost width of zones on its axis");
    }
    if (any && c->mhd) return fail(c, ADER_ERR_ARG, "non-periodic faces are built for Euler contexts");
    if (any && (c->guess || c->Dm))
        return fail(c, ADER_ERR_ARG, "non-periodic faces with the learned guess or dense output are not built");
    // drop the previous padded context
    if (c->inner) {
        c->inner->flag = nullptr;
        c->inner->stats = nullptr;
        ader_destroy(c->inner);
        c->inner = nullptr;
    }
    if (c->Upad) {
        cudaFree(c->Upad);
        c->Upad = nullptr;
    }
    for (int s = 0; s < 6; ++s) c->bc[s] = bc[s];
    for (int d = 0; d < 3; ++d) c->ghosts[d] = gh[d];
    if (!any) return ADER_OK;
    ader_grid gp = c->g;
    gp.nx += 2 * gh[0];
    gp.ny += 2 * gh[1];
    gp.nz += 2 * gh[2];
    ader_ctx* in = nullptr;
    if (int rc = ader_create(&gp, c->order, c->gamma, c->solver, c->flags, &in))
        return fail(c, rc, "context of the padded grid");
    cudaFree(in->flag);                        // reports through this context's flag and statistics
    cudaFree(in->stats);
    in->flag = c->flag;
    in->stats = c->stats;
    in->tiled = c->tiled;
    in->tol = c->tol;
    in->max_iter = c->max_iter;
    c->inner = in;
    if (c->src_kind != SOURCE_NONE) {
        const double par[3] = {c->src_par[0], c->src_par[1], c->src_par[2]};
        if (int rc = ader_set_source(in, c->src_kind == SOURCE_LINEAR ? ADER_SOURCE_LINEAR : ADER_SOURCE_GRAVITY, par))
            return fail(c, rc, in->err);
    }
    return cuda_check(c, cudaMalloc((void**)&c->Upad, (size_t)5 * (size_t)in->grid.n * sizeof(double)),
                      "cudaMalloc padded state");
}

int ader_set_predictor(ader_ctx* c, double tol, int max_iter) {
    if (!c) return ADER_ERR_ARG;
    if (tol < 0.0 || max_iter < 1 || max_iter > 1000) return fail(c, ADER_ERR_ARG, "tol >= 0, 1 <= max_iter <= 1000");
    c->tol = tol;
    c->max_iter = max_iter;
    if (c->inner) {
        c->inner->tol = tol;
        c->inner->max_iter = max_iter;
    }
    return ADER_OK;
}

int ader_predictor_stats(ader_ctx* c, unsigned long long* out3_host, void* stream) {
    if (!c || !out3_host) return ADER_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = cuda_check(c, cudaMemcpyAsync(out3_host, c->stats, 3 * sizeof(unsigned long long),
                                           cudaMemcpyDeviceToHost, st), "stats read");
    if (rc == ADER_OK) rc = cuda_check(c, cudaMemsetAsync(c->stats, 0, 3 * sizeof(unsigned long long), st), "memset");
    if (rc == ADER_OK) rc = cuda_check(c, cudaStreamSynchronize(st), "cudaStreamSynchronize");
    return rc;
}

int ader_set_source(ader_ctx* c, int kind, const double* params) {
    if (!c) return ADER_ERR_ARG;
    if (kind == ADER_SOURCE_NONE) {
        c->src_kind = SOURCE_NONE;
        if (c->inner) c->inner->src_kind = SOURCE_NONE;
        return ADER_OK;
    }
    if (kind != ADER_SOURCE_LINEAR && kind != ADER_SOURCE_GRAVITY) return fail(c, ADER_ERR_ARG, "unknown source kind");
    if (!params) return fail(c, ADER_ERR_ARG, "null source parameters");
    const int np = kind == ADER_SOURCE_LINEAR ? 1 : 3;
    double par[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < np; ++i) {
        if (!std::isfinite(params[i])) return fail(c, ADER_ERR_ARG, "non-finite source parameter");
        par[i] = params[i];
    }
    if (!c->Sb) {
        if (int rc = cuda_check(c, cudaMalloc(&c->Sb, (size_t)5 * (size_t)c->grid.n * c->rsize), "cudaMalloc source"))
            return rc;
    }
    c->src_kind = kind == ADER_SOURCE_LINEAR ? SOURCE_LINEAR : SOURCE_GRAVITY;
    for (int i = 0; i < 3; ++i) c->src_par[i] = par[i];
    if (c->inner) return ader_set_source(c->inner, kind, params) ? fail(c, ADER_ERR_CUDA, c->inner->err) : ADER_OK;
    return ADER_OK;
}

int ader_set_guess(ader_ctx* c, const float* params) {
    if (!c) return ADER_ERR_ARG;
    if (params && c->inner) return fail(c, ADER_ERR_ARG, "the learned guess with non-periodic faces is not built");
    if (params && c->order != 3) return fail(c, ADER_ERR_ARG, "the learned guess is built for third order");
    if (params && c->grid.n >= (1ll << 31)) return fail(c, ADER_ERR_ARG, "the learned guess takes up to 2^31 - 1 zones");
    if (params && !c->G) {
        const size_t N = (size_t)c->grid.n;
        const size_t bytes = (size_t)5 * (c->mhd ? 8 : 5) * N * sizeof(float);
        if (int rc = cuda_check(c, cudaMalloc((void**)&c->G, bytes), "cudaMalloc learned guess")) return rc;
        if (int rc = cuda_check(c, cudaMalloc((void**)&c->Glist, N * sizeof(int)), "cudaMalloc guess list")) return rc;
        if (int rc = cuda_check(c, cudaMalloc((void**)&c->Gact, N), "cudaMalloc guess flags")) return rc;
        if (int rc = cuda_check(c, cudaMalloc((void**)&c->Gcount, sizeof(unsigned)), "cudaMalloc guess count"))
            return rc;
        if (int rc = cuda_check(c, cudaMemset(c->Gcount, 0, sizeof(unsigned)), "cudaMemset guess count")) return rc;
    }
    c->guess = params;
    return ADER_OK;
}

int ader_trim_local_memory(size_t* kept_bytes) {
    size_t kept = 0;
    if (cudaDeviceGetLimit(&kept, cudaLimitStackSize) != cudaSuccess) return ADER_ERR_CUDA;
    if (kept_bytes) *kept_bytes = kept;
    if (cudaDeviceSynchronize() != cudaSuccess) return ADER_ERR_CUDA;
    return cudaDeviceSetLimit(cudaLimitStackSize, 1024) == cudaSuccess ? ADER_OK : ADER_ERR_CUDA;
}

int ader_test_bounded_wait(ader_ctx* c) {
    if (!c) return ADER_ERR_ARG;
    if (!c->guess) return fail(c, ADER_ERR_ARG, "no guess parameters set (ader_set_guess)");
    c->wait_test = true;
    return ADER_OK;
}

int ader_guess_eval(ader_ctx* c, const double* U, const double* Bface, double dt, float* G, void* stream) {
    if (!c) return ADER_ERR_ARG;
    if (!U || !G || !(dt > 0.0)) return fail(c, ADER_ERR_ARG, "null pointer or dt <= 0");
    if (!c->guess) return fail(c, ADER_ERR_ARG, "no guess parameters set (ader_set_guess)");
    if (int rc = check_bface(c, Bface)) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    StepArgs a = make_args(c, dt, nullptr, 2);
    a.Bface = Bface;
    a.guess = c->guess;
    a.G = G;
    c->wait_test = false;                     // one launch only
    if (c->fp32) {
        launch_recon<float>(a, U, st);
        if (launch_guess<float>(a, U, st, G) < 0) return fail(c, ADER_ERR_CUDA, "guess kernel set-up");
    } else {
        launch_recon<double>(a, U, st);
        if (launch_guess<double>(a, U, st, G) < 0) return fail(c, ADER_ERR_CUDA, "guess kernel set-up");
    }
    return cuda_check(c, cudaGetLastError(), "ader_guess_eval launch");
}

int ader_guess_count(ader_ctx* c, unsigned long long* out_host, void* stream) {
    if (!c || !out_host) return ADER_ERR_ARG;
    *out_host = 0;
    if (!c->Gcount) return ADER_OK;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned n = 0;
    int rc = cuda_check(c, cudaMemcpyAsync(&n, c->Gcount, sizeof(unsigned), cudaMemcpyDeviceToHost, st), "count read");
    if (rc == ADER_OK) rc = cuda_check(c, cudaStreamSynchronize(st), "cudaStreamSynchronize");
    if (rc == ADER_OK) *out_host = n;
    return rc;
}

int ader_guess_samples(ader_ctx* c, const double* U, const double* Bface, double dt, float* X, float* Y, int* ok,
                       void* stream) {
    if (!c) return ADER_ERR_ARG;
    if (!U || !X || !Y || !ok || !(dt > 0.0)) return fail(c, ADER_ERR_ARG, "null pointer or dt <= 0");
    if (int rc = check_bface(c, Bface)) return rc;
    if (c->order != 3 || c->fp32) return fail(c, ADER_ERR_ARG, "samples need a third-order FP64 context");
    cudaStream_t st = (cudaStream_t)stream;
    StepArgs a = make_args(c, dt, nullptr, 2);
    a.Bface = Bface;
    a.tol = c->tol > 0.0 ? c->tol : 1e-13;
    a.guess = nullptr;
    a.G = nullptr;
    launch_recon<double>(a, U, st);
    launch_guess_samples(a, U, X, Y, ok, st);
    return cuda_check(c, cudaGetLastError(), "ader_guess_samples launch");
}

int ader_sync_status(ader_ctx* c, void* stream) {
    if (!c) return ADER_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned h = 0;
    int rc = cuda_check(c, cudaMemcpyAsync(&h, c->flag, sizeof(unsigned), cudaMemcpyDeviceToHost, st), "flag read");
    if (rc == ADER_OK) rc = cuda_check(c, cudaStreamSynchronize(st), "cudaStreamSynchronize");
    if (rc != ADER_OK) return rc;
    if (h) {
        cudaMemsetAsync(c->flag, 0, sizeof(unsigned), st);
        cudaStreamSynchronize(st);
    }
    if (h & FLAG_NONFINITE) return fail(c, ADER_ERR_NONFINITE, "non-finite value in the updated state");
    if (h & FLAG_UNPHYSICAL) return fail(c, ADER_ERR_UNPHYSICAL, "rho <= 0 or P <= 0 in a zone");
    if (h & FLAG_TIMEOUT) return fail(c, ADER_ERR_TIMEOUT, "a bounded wait in a kernel ran out");
    if (h & FLAG_NOT_CONVERGED) return fail(c, ADER_ERR_NOT_CONVERGED, "predictor iteration cap reached");
    return ADER_OK;
}

int ader_step_host(ader_ctx* c, double* U_host, double* Bface_host, double cfl, double* dt_used_host) {
    if (!c) return ADER_ERR_ARG;
    if (!U_host) return fail(c, ADER_ERR_ARG, "U_host is null");
    if (Bface_host || c->mhd) return fail(c, ADER_ERR_ARG, "ader_step_host is built for Euler contexts only");
    const size_t bytes = (size_t)c->grid.n * 5 * sizeof(double);
    cudaStream_t st = 0;
    int rc = cuda_check(c, cudaMemcpyAsync(c->Ustage, U_host, bytes, cudaMemcpyHostToDevice, st), "H2D");
    if (rc == ADER_OK) rc = ader_max_dt(c, c->Ustage, nullptr, cfl, c->dt_dev, st);
    if (rc == ADER_OK) rc = ader_step_devdt(c, c->Ustage, nullptr, c->dt_dev, st);
    if (rc == ADER_OK) rc = cuda_check(c, cudaMemcpyAsync(U_host, c->Ustage, bytes, cudaMemcpyDeviceToHost, st), "D2H");
    if (rc == ADER_OK && dt_used_host)
        rc = cuda_check(c, cudaMemcpyAsync(dt_used_host, c->dt_dev, sizeof(double), cudaMemcpyDeviceToHost, st), "D2H dt");
    if (rc == ADER_OK) rc = cuda_check(c, cudaStreamSynchronize(st), "cudaStreamSynchronize");
    return rc;
}

// ----------------------------------------------------------------------------- dense output (Sec. VII)
static int mode_count(int order) { return order == 2 ? 5 : (order == 3 ? 15 : 35); }

int ader_set_dense_output(ader_ctx* c, int enable) {
    if (!c) return ADER_ERR_ARG;
    if (enable && c->inner) return fail(c, ADER_ERR_ARG, "dense output with non-periodic faces is not built");
    if (c->Dm) {
        if (int rc = cuda_check(c, cudaFree(c->Dm), "cudaFree dense modes")) return rc;
        c->Dm = nullptr;
    }
    c->dense_valid = false;
    if (!enable) return ADER_OK;
    const size_t bytes = (size_t)mode_count(c->order) * (c->mhd ? 8 : 5) * (size_t)c->grid.n * c->rsize;
    return cuda_check(c, cudaMalloc(&c->Dm, bytes), "cudaMalloc dense modes");
}

int ader_dense_output(ader_ctx* c, double tau, double* out, void* stream) {
    if (!c) return ADER_ERR_ARG;
    if (!out) return fail(c, ADER_ERR_ARG, "out is null");
    if (!(tau >= 0.0 && tau <= 1.0)) return fail(c, ADER_ERR_ARG, "tau must lie in [0, 1]");
    if (!c->Dm || !c->dense_valid) return fail(c, ADER_ERR_ARG, "no step has kept its modes (ader_set_dense_output)");
    cudaStream_t st = (cudaStream_t)stream;
    Trace t(c, "dense_output", st);
    launch_dense_eval(c->order, c->mhd ? 8 : 5, c->fp32, c->Dm, c->grid.n, tau, out, st);
    return cuda_check(c, cudaGetLastError(), "ader_dense_output launch");
}

}  // extern "C"

