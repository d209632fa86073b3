/*
 * ader.h -- C ABI of the GB300 (sm_103a) one-step ADER-WENO update on 3-D periodic meshes.
 *
 * The operation is the time step of Balsara, Meyer, Dumbser, Du & Xu,
 * "Efficient implementation of ADER schemes for Euler and MHD flows on
 * structured meshes" (arXiv:1006.2146):
 *   reconstruction (Sec. II.1), ADER-CG space-time predictor (Sec. II.2;
 *   modal Sec. IV, nodal Apps. A-C), space-time averaged fluxes at faces with
 *   the eigen-structure frozen at the face barycentre (Sec. II.3, Sec. V,
 *   App. D), and the single conservative update of Eq. 6.  The SSP-RK step
 *   of Eqs. 18-20 is provided for comparison on the same GPU.
 *
 * Conventions common to every entry point
 *   - Every array argument is a DEVICE pointer owned by the caller unless the
 *     name ends in _host.  The library owns only the scratch it allocates in
 *     ader_create and frees in ader_destroy; the step, dt and diagnostics
 *     entry points allocate nothing (the MLP entry points allocate their own
 *     workspace).
 *   - State layout (structure of arrays, FP64, x fastest):
 *       U[v][k][j][i], v = 0..4 = (rho, rho vx, rho vy, rho vz, eps),
 *       element (v, k, j, i) at U[((v*nz + k)*ny + j)*nx + i].
 *     eps is the total energy rho v^2/2 + P/(gamma-1) (+ B^2/8pi for MHD,
 *     Gaussian units, Eq. 3).
 *   - Boundaries are periodic in all three directions.  nx, ny, nz >= 1.
 *   - Work is enqueued asynchronously on the given CUDA stream (NULL = the
 *     legacy default stream); the call returns before the GPU finishes.
 *   - Return value: ADER_OK (0) or a negative ADER_ERR_* code.  The text of
 *     the last error of a context is returned by ader_last_error().  Errors
 *     detected on the device (a non-physical state: rho <= 0 or P <= 0, a
 *     non-finite value) set a device flag that ader_sync_status() reads.
 */
#ifndef ADER_GB300_H
#define ADER_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int nx, ny, nz;          /* zones per direction */
    double dx, dy, dz;       /* zone sizes */
} ader_grid;

/* Riemann solver at the faces (Sec. II.3, Eq. 56): HLL, or the linearized
 * solver with the eigen-structure of the flux Jacobian at the mean of the two
 * barycentre states (for MHD the seven-wave system; the edge electric fields
 * of Eq. 7 then use the same solver on the edge-averaged states). */
enum { ADER_HLL = 0, ADER_LINEARIZED = 1 };

/* Option flags for ader_create. */
enum {
    ADER_MHD = 1u << 0,                 /* ideal MHD with face-centred B and constrained transport */
    ADER_NODAL = 1u << 1,               /* nodal predictor (Apps. A-C); default modal (Sec. IV) */
    ADER_FP32_BULK = 1u << 2,           /* FP32 reconstruction/predictor/fluxes, FP64 update and reductions */
    ADER_CONVERGED_PREDICTOR = 1u << 4, /* iterate the predictor to tolerance instead of M-1 times */
    ADER_EMF_TRANSONIC = 1u << 5,       /* MHD: twice the dissipative term of Eq. 17 in the electric fields
                                           at transonic faces (Secs. II.3, V); transonic = a fast wave
                                           speed v -/+ c_f changes sign between the face's two states */
    ADER_POSITIVITY_FALLBACK = 1u << 6  /* FP64 only (with ADER_FP32_BULK: ADER_ERR_ARG): after each
                                           ader_step, the faces of zones left with rho <= 0 or P <= 0
                                           (MHD: P with the mean of the new face field) take the
                                           first-order HLL flux of the zone averages of step n and the
                                           zones around them are updated again (conservative; three
                                           passes).  MHD: every edge touching such a zone takes the
                                           first-order edge field (Eq. 7 from those fluxes) and the
                                           face field is advanced again from step n by Eq. 8 (div B
                                           kept).
                                           Costs a copy of U (5 x zones FP64) held by the context.  After
                                           the passes the step itself reports what is left: a non-finite
                                           zone value or (MHD) face value raises ADER_ERR_NONFINITE, a zone
                                           still non-physical ADER_ERR_UNPHYSICAL (read by
                                           ader_sync_status).  The paper names no positivity safeguard;
                                           this is an option. */
};

enum {
    ADER_OK = 0,
    ADER_ERR_ARG = -1,          /* invalid argument (null pointer, bad size/order/flag) */
    ADER_ERR_CUDA = -2,         /* a CUDA runtime call failed */
    ADER_ERR_UNPHYSICAL = -3,   /* device flag: rho <= 0 or P <= 0 met */
    ADER_ERR_NONFINITE = -4,    /* device flag: a NaN or Inf met */
    ADER_ERR_NOT_CONVERGED = -5, /* device flag: converged predictor hit its iteration cap */
    ADER_ERR_TIMEOUT = -6       /* device flag: a bounded wait inside a kernel ran out (the kernel
                                   stopped early; its outputs are incomplete) */
};

typedef struct ader_ctx ader_ctx;

/* Create a context for one grid.
 *   order  : 2, 3 or 4 (spatial and temporal order; L_S = 4/10/20 spatial
 *            modes, L = 5/15/35 space-time modes, Eqs. 10-16)
 *   gamma  : ratio of specific heats (> 1)
 *   solver : ADER_HLL or ADER_LINEARIZED
 *   flags  : bitwise OR of ADER_MHD, ADER_NODAL, ADER_FP32_BULK, ADER_EMF_TRANSONIC,
 *            ADER_POSITIVITY_FALLBACK (ADER_CONVERGED_PREDICTOR is
 *            rejected: use ader_set_predictor)
 * Allocates the device scratch for one step of this grid on the current
 * device.  *out receives the context; on failure *out is NULL. */
int ader_create(const ader_grid* g, int order, double gamma, int solver, unsigned flags, ader_ctx** out);

/* One ADER-WENO step of size dt (host value), in place on U (Eq. 6).
 * Euler: Bface must be NULL.  MHD (ADER_MHD): Bface[d][k][j][i] (3 x nz x ny x nx,
 * FP64) is the face-averaged normal field B_d on the face i_d - 1/2 of zone
 * (i, j, k) along d; the zone field is rebuilt from it every step (Sec. III,
 * face-B WENO) and it is advanced in place by constrained transport with
 * edge-averaged electric fields (Eqs. 7-8), which keeps its discrete
 * divergence unchanged to round-off.  U's energy includes B^2/8pi. */
int ader_step(ader_ctx* ctx, double* U, double* Bface, double dt, void* stream);

/* Same as ader_step with dt read on the device from dt_dev (one double), so
 * that a max_dt + step sequence needs no host round trip (graph capturable). */
int ader_step_devdt(ader_ctx* ctx, double* U, double* Bface, const double* dt_dev, void* stream);

/* CFL time step (reading of the paper's CFL rule, Secs. II.d and VI):
 *   dt = cfl / max over zones of sum_d (|v_d| + c_d) / dx_d,
 * c_d the sound speed (MHD: the fast speed with the zone field taken as the
 * mean of its two face values; Bface as for ader_step).  Written to dt_dev (one double, device).  Reduction
 * in FP64 with warp shuffles; FP32-bulk contexts compute each zone's signal speed in FP32 (dt then agrees
 * with the FP64 rule to about 1e-7 relative). */
int ader_max_dt(ader_ctx* ctx, const double* U, const double* Bface, double cfl, double* dt_dev, void* stream);

/* One SSP-RK step of the context's order (Eq. 18 for order 2, Eq. 19 for
 * order 3, Eq. 20 for order 4) with the same reconstruction and Riemann
 * solver and the App. D facial quadrature with every time mode zero.  MHD:
 * Bface advances with the same stage combinations, its operator being
 * -curl E from the stage's edge fields (the rate whose Euler step is Eq. 8),
 * so every stage keeps the discrete div B.  U and Bface as for ader_step. */
int ader_rk_step(ader_ctx* ctx, double* U, double* Bface, double dt, void* stream);

/* End-to-end step through host memory: copies U_host to the device, runs
 * ader_max_dt (cfl) then ader_step, copies U back and returns the dt used in
 * *dt_used_host.  Synchronous.  U_host should be pinned for full speed.
 * Euler contexts only. */
int ader_step_host(ader_ctx* ctx, double* U_host, double* Bface_host, double cfl, double* dt_used_host);

/* Conservation and divergence diagnostics (FP64, deterministic order).
 * Euler: totals of the five conserved variables -> totals_dev[0..4].
 * MHD: totals_dev[0..4] as above, [5..7] totals of the face fields Bx, By, Bz,
 * [8] the largest |div B| of a zone (sum over d of the face difference over
 * dx_d, the quantity Eq. 8 keeps constant) over (largest |B| on a face /
 * min(dx, dy, dz)); 0 when B vanishes.  totals_dev is device memory of 5
 * (Euler) or 9 (MHD) doubles. */
int ader_diagnostics(ader_ctx* ctx, const double* U, const double* Bface, double* totals_dev, void* stream);

/* Synchronise the stream and turn the device error flag into a return code
 * (ADER_OK, ADER_ERR_UNPHYSICAL, ADER_ERR_NONFINITE, ADER_ERR_TIMEOUT, ADER_ERR_NOT_CONVERGED);
 * clears the flag. */
int ader_sync_status(ader_ctx* ctx, void* stream);

/* Number of kernel launches the last ader_step / ader_rk_step enqueued. */
int ader_launches_per_step(const ader_ctx* ctx);

/* Per-kernel timing (tracing).  While enabled, every kernel the context
 * enqueues is bracketed by CUDA events on its stream.  ader_profile_read
 * synchronises the events, writes for up to `cap` kernel names their launch
 * count and summed device time (ms) and returns the number of names (or a
 * negative code); names are static strings owned by the library.  enable = 0
 * stops recording; ader_profile_reset clears the totals. */
int ader_profile(ader_ctx* ctx, int enable);
int ader_profile_reset(ader_ctx* ctx);
int ader_profile_read(ader_ctx* ctx, const char** names, int* launches, double* ms, int cap);

/* Converged predictor.  tol > 0: iterate the ADER-CG predictor of every zone
 * until the largest change of an evolutionary mode is below tol times the
 * zone's largest |w_1| (at most max_iter times; reaching the cap raises
 * ADER_ERR_NOT_CONVERGED); tol = 0 restores the paper's M-1 iterations
 * (Secs. IV.1-IV.3).  ader_predictor_stats writes {sum of iterations over
 * zones and steps, largest count, zones capped} to out3_host and clears them
 * (synchronises the stream). */
int ader_set_predictor(ader_ctx* ctx, double tol, int max_iter);

/* Launch layout of the Euler step at orders 2 and 3 (Sec. II's per-zone
 * pipeline: predictor,
 * face quadrature, Riemann solve, Eq. 6).  on = 1 (the default): a block owns
 * a 32 x 4 tile of columns and marches through z; the six face sides of each
 * zone stay in shared memory, every face inside the tile is solved once, and
 * only the tile's boundary sides pass through memory.  on = 0: every zone
 * writes its face data to the context's scratch and a second pass solves the
 * faces.  Both give the same numbers bit for bit in FP64 (in FP32 bulk to
 * FP32 rounding: the compiler may contract the predictor's multiply-adds
 * differently in the two kernels); MHD contexts and order 4
 * always take the second layout (the edge fields need the face data of four
 * zones; the fourth-order predictor's cost dwarfs the face data's traffic).
 * on = 1 also computes the third-order cross moments of the reconstruction
 * (Euler and MHD) in shared-memory tiles of 32 x 8 columns where nx is a
 * multiple of 32 and ny of 8, each WENO term of a position once for all the
 * zones that use it; on = 0 takes the per-zone kernel, with the same bits in
 * FP64 (FP32 to FP32 rounding).
 * ADER_ERR_ARG for a NULL context. */
int ader_set_tiled(ader_ctx* ctx, int on);

/* Box faces (Euler contexts).  bc[6] = {x-, x+, y-, y+, z-, z+}, each
 * ADER_BC_PERIODIC (the default), ADER_BC_OUTFLOW or ADER_BC_REFLECTIVE; an
 * axis is periodic on both faces or on neither.  The paper's tests with walls
 * and open sides (Sec. VIII) state no boundary treatment; this is the usual
 * ghost-zone one: G ghost zones (3 at orders 2-3, 4 at order 4, a step's reach)
 * across every non-periodic face, an outflow ghost copying the nearest interior
 * zone, a reflecting ghost the mirror-image zone with the normal momentum
 * negated.  With a non-periodic face, ader_step / ader_step_devdt /
 * ader_step_host fill a padded state from U (held by the context: 5 x padded
 * zones FP64, plus the padded grid's scratch), step it and copy its interior
 * back to U; ader_max_dt and ader_diagnostics read U as before.  The converged
 * predictor, source terms, FP32 bulk, the positivity fallback and the launch
 * layout carry over.  ADER_ERR_ARG for an unknown code, an axis periodic on one
 * face only, a reflecting axis shorter than G zones, an MHD context, or a
 * context with the learned guess or dense output; ader_rk_step then returns
 * ADER_ERR_ARG (not built).  ADER_ERR_CUDA if an allocation fails. */
#define ADER_BC_PERIODIC 0
#define ADER_BC_OUTFLOW 1
#define ADER_BC_REFLECTIVE 2
int ader_set_boundary(ader_ctx* ctx, const int* bc);
int ader_predictor_stats(ader_ctx* ctx, unsigned long long* out3_host, void* stream);

/* Non-stiff source term S(U) of Eq. 4 (Sec. II; orders 2-4, modal and
 * nodal).  The paper carries a general S through the predictor (Eqs. 30, 34,
 * 36, 43, 45, 52; A.4, B.2-B.3, C.2-C.3) and the update (Eq. 6 with S-bar of
 * Eqs. 35, 44, 53; A.7, B.6, C.6) without naming one; two models are built:
 *   ADER_SOURCE_LINEAR:  S = -k U on the five hydrodynamic variables,
 *                        params[0] = k;
 *   ADER_SOURCE_GRAVITY: S = (0, rho g, rho v . g), params[0..2] = g.
 * The face field of MHD gets no source (Eq. 8 is unchanged).  The predictor
 * evaluates the source at its nodes each iteration; S-bar comes from the
 * source polynomial of the final iterate.  params is a host array (1 or 3
 * doubles, copied); ADER_SOURCE_NONE (params may be NULL) removes the source.
 * The first source allocates a per-zone buffer (5 x zones, bulk precision).
 * Returns ADER_ERR_ARG for an unknown kind or non-finite parameters.  ader_rk_step refuses a context with a source, and the
 * learned-guess samples (ader_guess_samples) are taken without it. */
#define ADER_SOURCE_NONE 0
#define ADER_SOURCE_LINEAR 1
#define ADER_SOURCE_GRAVITY 2
int ader_set_source(ader_ctx* ctx, int kind, const double* params);

/* Dense output inside a step (Sec. VII: the predictor's space-time polynomial
 * gives the solution at any time within the step, which is what the finer
 * levels of an adaptive mesh, taking shorter steps, need from a coarse zone).
 * ader_set_dense_output(ctx, 1) makes every later ader_step / ader_step_devdt
 * keep all L space-time modes of each zone's predictor (L = 5 / 15 / 35 at
 * orders 2 / 3 / 4; L x nvar x zones values of the bulk precision, allocated
 * and held by the context); 0 frees them.  ADER_ERR_CUDA if the allocation
 * fails.  SSP-RK steps keep nothing. */
int ader_set_dense_output(ader_ctx* ctx, int enable);
/* Writes, for the last step that kept its modes, the LS spatial modes (LS = 4
 * / 10 / 20) of every zone's polynomial at time t^n + tau dt, 0 <= tau <= 1:
 * out[(s*nvar + v)*zones + zone], FP64 device memory, s = 0..LS-1 the spatial
 * modes in the order of Eqs. 14-16 (s = 0 is the zone average; for MHD the
 * field variables are the zone field's modes).  Asynchronous on the stream.
 * ADER_ERR_ARG for tau outside [0, 1], a NULL out, or no step since enabling. */
int ader_dense_output(ader_ctx* ctx, double tau, double* out, void* stream);

/* Learned initial guess (third order; the paper has no learned component and
 * starts its Picard iteration of Sec. IV from zero).  params (device, FP32,
 * layout and size from ader_mlp_shape) is an MLP mapping a zone's normalised
 * spatial modes and Courant numbers to its evolutionary modes; each step then
 * runs two more kernels: one lists the zones that carry slopes (the guess of
 * a zone whose slope magnitude is below 1e-12 is exactly zero), the other
 * runs the network on those zones only, and the predictor starts from the
 * guess instead of zero.  The first non-NULL call allocates the per-zone
 * buffers (the guess, 5 x nvar x zones FP32; the list and flags, 5 bytes per
 * zone; held by the context); NULL disables the guess.  Grids of 2^31 zones
 * or more return ADER_ERR_ARG.  The pointer is kept, not copied: keep the buffer alive while the
 * context uses it.  With the fixed iteration count the guess changes the
 * result; with ader_set_predictor's tolerance it only changes the work. */
int ader_set_guess(ader_ctx* ctx, const float* params);
/* The guess alone: reconstructs (U, Bface) and writes every zone's guessed
 * evolutionary modes to G (device, 5 x nvar x zones FP32, G[(j*nvar + v)*zones
 * + zone] = u_{11+j} of variable v) with the kernel the step uses: the three
 * layers on the tensor cores (tcgen05, FP16 operands, FP32 accumulation).
 * Needs ader_set_guess first.  Asynchronous on the stream. */
int ader_guess_eval(ader_ctx* ctx, const double* U, const double* Bface, double dt, float* G, void* stream);
/* Local memory of the CUDA context (runtime housekeeping; no counterpart in
 * the paper).  The context keeps, for every thread of every later launch, the
 * largest per-thread stack a kernel has needed (the FP64 fourth-order
 * predictor needs about 5 KB); kernels with smaller frames that spill then
 * run in that wider layout, the FP32 fourth-order predictor about 25% slower.
 * This sets the context's stack limit back to 1 KB per thread
 * (cudaDeviceSetLimit(cudaLimitStackSize)), freeing the rest; the next launch
 * that needs more grows it again.  *kept_bytes (host, may be NULL) receives
 * the per-thread stack size held before the call.  Synchronises the device;
 * not during a stream capture.  ADER_ERR_CUDA if the runtime refuses. */
int ader_trim_local_memory(size_t* kept_bytes);
/* Test of the tensor-core kernel's bounded waits (failure detection; no
 * counterpart in the paper).  Arms the context's next learned-guess launch
 * (ader_guess_eval, or a step with a guess): that launch issues no MMA for its
 * first layer, so that nothing ever completes the barrier it waits on; after
 * 1024 tries the wait gives up, the kernel raises ADER_ERR_TIMEOUT (read by
 * ader_sync_status), frees its tensor memory and returns, leaving its guess
 * output unwritten.  The arming holds for one launch.  ADER_ERR_ARG for a NULL
 * context or one without guess parameters. */
int ader_test_bounded_wait(ader_ctx* ctx);
/* The number of zones the network ran on in the context's last guess launch
 * (the zones with slopes), to *out_host; synchronises the stream.  0 before
 * the first launch or without a guess. */
int ader_guess_count(ader_ctx* ctx, unsigned long long* out_host, void* stream);
int ader_mlp_shape(int mhd, int* n_in, int* n_hidden, int* n_out, long long* n_params);

/* Training data: for every zone of (U, Bface), the MLP features X (n x n_in)
 * and the normalised evolutionary modes Y (n x n_out) of the converged FP64
 * modal predictor started from zero (tolerance of ader_set_predictor, 1e-13
 * if unset).  Features: the zone's slopes (modes w2..w10 over the variable
 * scales) divided by their largest magnitude g; the zone means of momentum
 * (and field) over their scales; the three Courant numbers; and g.  Targets
 * are divided by g as well.  ok[z] = 0 marks a zone to skip: non-physical,
 * uniform to round-off (g <= 1e-12, whose guess is zero by construction) or
 * capped; its rows
 * are left unwritten.  Needs a third-order FP64 context.  All pointers are
 * device pointers. */
int ader_guess_samples(ader_ctx* ctx, const double* U, const double* Bface, double dt, float* X, float* Y, int* ok,
                       void* stream);

/* MLP training on the GPU with the library's own kernels (FP32 GEMM, GELU,
 * Adam; mean-squared error).  X, Y: device samples (n rows); params:
 * device parameters, updated in place (initialise them first);
 * loss_per_epoch_host: optional host array of `epochs` doubles.  Allocates
 * and frees its own workspace.  Synchronous. */
int ader_mlp_train(const float* X, const float* Y, long long n, int mhd, int epochs, int batch, float lr,
                   unsigned long long seed, float* params, double* loss_per_epoch_host, void* stream);

/* Mean-squared-error loss and its gradient (device grad, size n_params) on n
 * samples: the training kernels' forward and backward pass, exposed for
 * checking them.  Synchronous. */
int ader_mlp_grad(const float* params, const float* X, const float* Y, long long n, int mhd, float* grad,
                  double* loss_host, void* stream);

const char* ader_last_error(const ader_ctx* ctx);
void ader_destroy(ader_ctx* ctx);

/* ---- Batched problems (many independent grids in one captured step) ----
 * Each problem is the periodic problem of Eqs. 4-8 on its own grid, with its
 * own order, gamma, solver and flags; the batch advances all of them by one
 * ADER step (Eq. 6, and Eq. 8 for MHD) per call.  The paper has no batched
 * mode: it runs one problem at a time.  Problems must use ADER_FP32_BULK (FP32
 * reconstruction, predictor and fluxes; FP64 state, update and dt) and the
 * fixed iteration count of the predictor.
 * Problems of the same order, physics, form and solver form a group; each
 * phase of a group is one persistent launch over all its problems, groups run
 * concurrently, and a step is replayed from a CUDA graph captured on the first
 * call (captured again when the state pointers, dt buffer or CFL change).
 *   ader_batch_create: n problems (1..ADER_BATCH_MAX), arrays of n entries.
 *     Allocates all scratch; nothing is allocated by the step calls.
 *   ader_batch_tune: optional; times each (group, phase) over block sizes
 *     64/128/256 and persistent grid sizes on private copies of the given
 *     states (allocated and freed inside the call) and keeps the fastest.
 *   ader_batch_step: U[p] (device, 5 x zones, in/out), Bface[p] (device,
 *     3 x zones for MHD problems, else ignored), dt_dev[p] (device, n doubles).
 *   ader_batch_advance: dt_dev[p] = cfl / max over zones of sum_d (|v_d| +
 *     c_d) / dx_d for each problem (written to dt_dev, device, n doubles; NULL
 *     uses an internal buffer; signal speeds in FP32, maximum in FP64), then
 *     the step with it; one graph.
 *   ader_batch_status: synchronises the stream; codes_host[p] (n ints, may be
 *     NULL) gets each problem's code; returns the first non-OK code.
 *   ader_batch_tuning: writes (group, phase, threads, blocks) quadruples
 *     (blocks 0 = one block per `threads` zones) to out_host (cap ints);
 *     returns the number of quadruples.
 * The pointer arrays are host arrays; the pointers they hold are device
 * pointers and stay owned by the caller. */
#define ADER_BATCH_MAX 4096
typedef struct ader_batch ader_batch;
int ader_batch_create(int n, const ader_grid* grids, const int* orders, const double* gammas, const int* solvers,
                      const unsigned* flags, ader_batch** out);
int ader_batch_tune(ader_batch* b, double* const* U, double* const* Bface, void* stream);
int ader_batch_step(ader_batch* b, double* const* U, double* const* Bface, const double* dt_dev, void* stream);
int ader_batch_advance(ader_batch* b, double* const* U, double* const* Bface, double cfl, double* dt_dev,
                       void* stream);
int ader_batch_status(ader_batch* b, int* codes_host, void* stream);
int ader_batch_tuning(const ader_batch* b, int* out_host, int cap);
int ader_batch_groups(const ader_batch* b);
const char* ader_batch_last_error(const ader_batch* b);
void ader_batch_destroy(ader_batch* b);

/* CFL time step that allocates nothing (the paper has no counterpart: this is
 * a deployment variant of ader_max_dt).  For callers that cannot call
 * cudaMalloc -- inside someone else's stream capture, real-time loops with a
 * fixed memory budget, hosts that forbid device allocation after start-up --
 * it needs no context and keeps its scratch in a file-scope device array of
 * the library (512 KB; one per device that loads the library, held until the
 * process exits).
 *   g, gamma : grid and ratio of specific heats, as for ader_create (Euler)
 *   U        : device state, layout as above (read only)
 *   cfl      : Courant number (> 0); dt = cfl / max_zones sum_d (|v_d| + a) / dx_d
 *   dt_dev   : device output, one double
 * Grids larger than ADER_STATIC_MAX_ZONES zones return ADER_ERR_ARG.  The
 * first call on a device looks up the array's device address (with that
 * device current); make that first call before any stream capture.  All calls
 * share the array, so calls that overlap on the GPU race: serialise them.
 * Returns ADER_OK, ADER_ERR_ARG or ADER_ERR_CUDA.  A zone with rho <= 0,
 * P <= 0 or a non-finite value has no signal speed: *dt_dev is then a quiet
 * NaN (a step taken with it turns the state non-finite, which
 * ader_sync_status reports). */
#define ADER_STATIC_MAX_ZONES 268435456LL
int ader_max_dt_static(const ader_grid* g, double gamma, const double* U, double cfl, double* dt_dev, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* ADER_GB300_H */
