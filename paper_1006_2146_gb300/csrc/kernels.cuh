// Launch interface shared by the kernel translation units and the C ABI.
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace ader {

enum { FORM_MODAL = 0, FORM_NODAL = 1 };
enum { SOLVER_HLL = 0, SOLVER_LINEARIZED = 1 };

// Everything a step's kernels need, passed by value.
struct StepArgs {
    Grid grid;
    int order;          // 2, 3, 4
    int form;           // FORM_MODAL / FORM_NODAL
    int solver;         // SOLVER_HLL / SOLVER_LINEARIZED
    int fp32;           // 1: FP32 bulk arithmetic
    int n_iter;         // predictor iterations (order - 1 by default; 0 = spatial only, used by SSP-RK)
    double tol;         // > 0: converged predictor (iterate to tolerance, at most max_iter times)
    int max_iter;
    unsigned long long* stats;   // converged predictor: [0] sum of iterations, [1] max, [2] zones capped
    const float* guess; // learned initial guess: packed MLP weights (order 3), or null
    float* G;           // learned initial guess per zone: u_11..u_15 (5 x NV x N, FP32), written by the
                        // guess kernel and read by the predictor; null = start from zero
    int* Glist;         // with a guess: the zones that carry slopes (the only ones the network runs on),
    unsigned* Gcount;   // their number (device), and a per-zone flag the predictor reads before G;
    unsigned char* Gact;    // a zone without the flag starts from zero (its guess is exactly zero)
    double gamma;
    double dx[3];
    double idx[3];      // 1 / dx, computed once on the host
    double gm1;         // gamma - 1
    float gamma_f, gm1_f, idx_f[3];   // FP32 copies for the FP32-bulk kernels (no FP64 work per zone)
    double dt;          // used when dt_dev is null
    const double* dt_dev;
    void* S1;           // 1-D WENO moments          (R)
    void* S2;           // cross moments             (R)
    void* S3;           // face-side data             (R)
    unsigned* flag;     // device error flag
    int mhd;            // 1: ideal MHD (8 variables, face-centred B)
    const double* Bface; // MHD: face field B_d on faces i_d - 1/2 (3 x N), read
    void* ZB;           // MHD: zone-averaged B from the face-B WENO (3 x N, R)
    void* E;            // MHD: edge EMFs Ex, Ey, Ez (3 x N, R)
    const float* Uf;    // FP32 bulk: the state rounded to FP32 once per step (5 x N), read by the WENO
    int src_kind;       // SOURCE_NONE / SOURCE_LINEAR / SOURCE_GRAVITY
    double src_par[3];  // k (linear) or g (gravity)
    void* Sb;           // with a source: dt S-bar of Eq. 6 per zone (5 x N, R), written by the predictor
    void* modes_out;    // dense output: every space-time mode of the predictor (L x NV x N, R), or null
    int emf_transonic;  // MHD: twice the dissipative term of the EMF fluxes at transonic faces
    int defer_nonfinite;  // the positivity fallback checks the updated state itself (after its passes)
    int wait_test;      // the learned-guess kernel's test of its bounded waits (ader_test_bounded_wait)
    int tiled;          // Euler, orders 2-3: predictor and face solves per 2.5-D tile (k_pf_tile), fluxes
                        // stored once per face in S1; 0: face data of every zone through S3 (MHD, order 4)
};

// gamma, gamma - 1 and 1 / dx_d in the bulk precision R
template <class R> ADER_DEV R arg_gamma(const StepArgs& a) {
    if constexpr (sizeof(R) == 4) return a.gamma_f; else return R(a.gamma);
}
template <class R> ADER_DEV R arg_gm1(const StepArgs& a) {
    if constexpr (sizeof(R) == 4) return a.gm1_f; else return R(a.gm1);
}
template <class R> ADER_DEV R arg_idx(const StepArgs& a, int d) {
    if constexpr (sizeof(R) == 4) return a.idx_f[d]; else return R(a.idx[d]);
}
// fills the derived fields from gamma and dx
inline void finish_args(StepArgs& a) {
    a.gm1 = a.gamma - 1.0;
    a.gamma_f = (float)a.gamma;
    a.gm1_f = (float)a.gm1;
    for (int d = 0; d < 3; ++d) {
        a.idx[d] = 1.0 / a.dx[d];
        a.idx_f[d] = (float)a.idx[d];
    }
}

// Number of R values per zone in each scratch array.
inline int nvar(int mhd) { return mhd ? 8 : 5; }
inline int s1_per_zone(int order, int mhd) { return nvar(mhd) * 3 * (order - 1); }
inline int s2_per_zone(int order, int mhd) { return order == 2 ? 0 : nvar(mhd) * (order == 3 ? 3 : 10); }
// face-side values per side: u_b, <u>, <F> (NV each) and, for MHD, 4 edges x (<u_c>, <F_c>)
ADER_DEV constexpr int side_values(int nv) { return 3 * nv + (nv == 8 ? 8 : 0); }
// MHD with the linearized solver also keeps every edge's full averaged state: a second block of
// 6 sides x 4 edges x 8 components after the 6 x side_values(8) of the first
constexpr int EDGE_STATE_VALUES = 4 * 8;
inline int s3_per_zone(int mhd, int linearized = 0) {
    return 6 * side_values(nvar(mhd)) + (mhd && linearized ? 6 * EDGE_STATE_VALUES : 0);
}

template <class R> int launch_recon(const StepArgs& a, const double* U, cudaStream_t st);
// out[i] = (float)U[i], i < count (the FP32 copy of the state the FP32 WENO reads)
int launch_to_f32(float* out, const double* U, long long count, cudaStream_t st);
// FP64: first-order fluxes on the faces of zones left non-physical, conservative re-update; MHD (Bold: the face
// field of step n) also first-order edge fields around them and Eq. 8 again (positivity.cu)
int launch_positivity_fallback(const StepArgs& a, double* U, const double* Uold, const double* Bold,
                               unsigned char* mark, double c_host, bool use_dt_dev, cudaStream_t st);
// dense output: the LS spatial modes at time tau of the space-time modes kept by a step (dense.cu)
int launch_dense_eval(int order, int nv, bool fp32, const void* modes, long long N, double tau, double* out,
                      cudaStream_t st);
template <int ORDER, int NV, class R> int launch_predict_faces_nv(const StepArgs& a, const double* U, cudaStream_t st);
// out = base + c * L(U) with L = -sum_d (F(i+1/2) - F(i-1/2)) / dx_d from the face data in S3;
// c = c_host, multiplied by *a.dt_dev when use_dt_dev; base may equal out (in place) or be null (out = c L).
template <class R> int launch_flux_update(const StepArgs& a, double* out, const double* base, double c_host,
                                          bool use_dt_dev, cudaStream_t st);
// out = sum_i c[i] X[i], i < n (n <= 6)
int launch_lincomb(double* out, int n, const double* const* X, const double* c, long long count, cudaStream_t st);

// fp32: per-zone signal speeds in FP32 (FP32-bulk contexts); the reduction and dt are FP64 either way
int launch_max_dt(const Grid& g, const double* U, const double* Bf, double gamma, const double dx[3], double cfl,
                  double* dt_dev, unsigned long long* scratch, unsigned* flag, bool fp32, cudaStream_t st);
// MHD: edge EMFs from the face data in S3, then Eq. 8 on Bf (in place) with step c_host (x *dt_dev)
template <class R> int launch_emf_ct(const StepArgs& a, double* Bf, double c_host, bool use_dt_dev, cudaStream_t st);
int launch_guess_samples(const StepArgs& a, const double* U, float* X, float* Y, int* ok, cudaStream_t st);
// learned guess of every zone into a.G (order 3; after launch_recon)
template <class R> int launch_guess(const StepArgs& a, const double* U, cudaStream_t st, float* Gzero);
// non-periodic box faces (boundary.cu): the padded state gp with ghost zones per the face rules, and back
int launch_fill_ghosts(const Grid& g, const Grid& gp, const int bc[6], const int gh[3], const double* U, double* Up,
                       cudaStream_t st);
int launch_copy_interior(const Grid& g, const Grid& gp, const int gh[3], const double* Up, double* U, cudaStream_t st);
int launch_totals(const Grid& g, const double* U, const double* Bf, const double dx[3], double* totals_dev,
                  double* partial, int nblocks, cudaStream_t st);

}  // namespace ader
