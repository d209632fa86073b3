// A-posteriori positivity fallback for the FP64 step (Euler and MHD) (an option of this library; the paper names
// no safeguard).  After the update, zones whose average is non-physical (rho <= 0, P <= 0 or not finite)
// are marked; every face of a marked zone gets the first-order HLL flux of the two zone averages of U^n
// (Eq. 56 with the zone averages as barycentre and averaged states), written over the stored face flux;
// every zone next to a marked one is then updated again from U^n with the stored fluxes, which both
// zones of a face share, so the step stays conservative.  MHD: every edge touching a marked zone also
// takes the first-order electric field, and the faces around those edges are advanced again from the
// face field of step n (Eq. 8; div B is kept).  Three passes, the marks accumulating; a pass with no mark
// changes nothing.  The update leaves the non-finite check to the fallback, which mends such
// zones like non-physical ones and checks the state (and, for MHD, the face field) after its passes.
#include "kernels.cuh"
#include "riemann.cuh"
#include "step_kernels.cuh"

namespace ader {

namespace {

// rho <= 0, P <= 0 or not finite; MHD: P with the mean of the zone's two new face values per direction
template <int NV>
ADER_DEV bool unphysical(const Grid& g, const double* U, const double* Bf, long long z, double gm1) {
    const long long N = g.n;
    const double rho = U[z];
    const double m1 = U[N + z], m2 = U[2 * N + z], m3 = U[3 * N + z];
    double e = U[4 * N + z] - 0.5 * (m1 * m1 + m2 * m2 + m3 * m3) / rho;
    if constexpr (NV == 8) {
        int i, j, k;
        zone_ijk(g, z, i, j, k);
        const double bx = 0.5 * (Bf[z] + Bf[nbr_along(g, z, i, j, k, 0, 1)]);
        const double by = 0.5 * (Bf[N + z] + Bf[N + nbr_along(g, z, i, j, k, 1, 1)]);
        const double bz = 0.5 * (Bf[2 * N + z] + Bf[2 * N + nbr_along(g, z, i, j, k, 2, 1)]);
        e = e - (bx * bx + by * by + bz * bz) / (8.0 * 3.141592653589793);
    }
    return !(rho > 0.0) || !(gm1 * e > 0.0);
}

template <int NV>
__global__ void __launch_bounds__(256) k_pos_mark(Grid g, const double* __restrict__ U, const double* __restrict__ Bf,
                                                  double gm1, unsigned char* __restrict__ mark) {
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (z < g.n && unphysical<NV>(g, U, Bf, z, gm1)) mark[z] = 1;
}

// the zone states of step n: U^n and, for MHD, the zone field of the face-B reconstruction (ZB)
template <int NV>
ADER_DEV Vec<NV, double> state_n(const StepArgs& a, const double* Uold, long long z) {
    const long long N = a.grid.n;
    Vec<NV, double> u;
#pragma unroll
    for (int v = 0; v < 5; ++v) u[v] = Uold[v * N + z];
    if constexpr (NV == 8) {
        const double* ZB = (const double*)a.ZB;
#pragma unroll
        for (int c = 0; c < 3; ++c) u[5 + c] = ZB[c * N + z];
    }
    return u;
}

template <int D, int NV>
ADER_DEV void first_order_face(const StepArgs& a, const double* Uold, long long z, long long zp) {
    const long long N = a.grid.n;
    FaceSide<NV, double> L, Rt;
    L.ub = L.avg = state_n<NV>(a, Uold, z);
    Rt.ub = Rt.avg = state_n<NV>(a, Uold, zp);
    L.F = flux<D>(L.ub, a.gm1);
    Rt.F = flux<D>(Rt.ub, a.gm1);
    const Vec<NV, double> f = riemann_hll<D>(L, Rt, a.gamma, a.gm1);
    double* F = (double*)a.S1;
#pragma unroll
    for (int v = 0; v < 5; ++v) F[(D * 5 + v) * N + z] = f[v];
}

// the three upper faces of zone z (stored at z) that touch a marked zone
template <int NV>
__global__ void __launch_bounds__(128) k_pos_faces(StepArgs a, const double* __restrict__ Uold,
                                                   const unsigned char* __restrict__ mark) {
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= a.grid.n) return;
    int i, j, k;
    zone_ijk(a.grid, z, i, j, k);
    const long long zx = nbr_along(a.grid, z, i, j, k, 0, 1), zy = nbr_along(a.grid, z, i, j, k, 1, 1),
                    zz = nbr_along(a.grid, z, i, j, k, 2, 1);
    const bool mz = mark[z];
    if (mz || mark[zx]) first_order_face<0, NV>(a, Uold, z, zx);
    if (mz || mark[zy]) first_order_face<1, NV>(a, Uold, z, zy);
    if (mz || mark[zz]) first_order_face<2, NV>(a, Uold, z, zz);
}

// zones with a marked zone among themselves and their six face neighbours: Eq. 6 again from U^n
__global__ void __launch_bounds__(128) k_pos_update(StepArgs a, double* U, const double* __restrict__ Uold,
                                                    const unsigned char* __restrict__ mark, double c_host,
                                                    int use_dt_dev) {
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= a.grid.n) return;
    int i, j, k;
    zone_ijk(a.grid, z, i, j, k);
    bool near = mark[z];
#pragma unroll
    for (int D = 0; D < 3; ++D) {
        near |= mark[nbr_along(a.grid, z, i, j, k, D, 1)] != 0;
        near |= mark[nbr_along(a.grid, z, i, j, k, D, -1)] != 0;
    }
    if (near) zone_flux_update_stored<double>(a, U, Uold, c_host, use_dt_dev, z);
}

// MHD: the first-order electric field of every edge that touches a marked zone (Eq. 7's mean of the four
// adjacent faces' fluxes, each the first-order HLL flux of the zone states of step n: the edge averages of
// a piecewise-constant state are its zone averages), written over the step's edge field in E.  Zone z
// owns its three upper edges, as in zone_emf: Ex on (j+1/2, k+1/2), Ey on (i+1/2, k+1/2), Ez on
// (i+1/2, j+1/2).
template <int D>
ADER_DEV Vec<8, double> first_order_flux(const StepArgs& a, const double* Uold, long long zl, long long zr) {
    FaceSide<8, double> L, Rt;
    L.ub = L.avg = state_n<8>(a, Uold, zl);
    Rt.ub = Rt.avg = state_n<8>(a, Uold, zr);
    L.F = flux<D>(L.ub, a.gm1);
    Rt.F = flux<D>(Rt.ub, a.gm1);
    return riemann_hll<D>(L, Rt, a.gamma, a.gm1);
}

__global__ void __launch_bounds__(128) k_pos_emf(StepArgs a, const double* __restrict__ Uold,
                                                 const unsigned char* __restrict__ mark) {
    const Grid& g = a.grid;
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= g.n) return;
    int i, j, k;
    zone_ijk(g, z, i, j, k);
    const long long zx = nbr(g, i, j, k, 1, 0, 0), zy = nbr(g, i, j, k, 0, 1, 0), zz = nbr(g, i, j, k, 0, 0, 1);
    const long long zxy = nbr(g, i, j, k, 1, 1, 0), zxz = nbr(g, i, j, k, 1, 0, 1), zyz = nbr(g, i, j, k, 0, 1, 1);
    const bool m0 = mark[z], mx = mark[zx], my = mark[zy], mz = mark[zz];
    double* E = (double*)a.E;
    if (m0 || mx || my || mark[zxy]) {          // Ez = (-F7 - F7 + G6 + G6) / 4
        const double f1 = first_order_flux<0>(a, Uold, z, zx)[6], f2 = first_order_flux<0>(a, Uold, zy, zxy)[6];
        const double g1 = first_order_flux<1>(a, Uold, z, zy)[5], g2 = first_order_flux<1>(a, Uold, zx, zxy)[5];
        E[2 * g.n + z] = 0.25 * (-f1 - f2 + g1 + g2);
    }
    if (m0 || mx || mz || mark[zxz]) {          // Ey = (F8 + F8 - H6 - H6) / 4
        const double f1 = first_order_flux<0>(a, Uold, z, zx)[7], f2 = first_order_flux<0>(a, Uold, zz, zxz)[7];
        const double h1 = first_order_flux<2>(a, Uold, z, zz)[5], h2 = first_order_flux<2>(a, Uold, zx, zxz)[5];
        E[g.n + z] = 0.25 * (f1 + f2 - h1 - h2);
    }
    if (m0 || my || mz || mark[zyz]) {          // Ex = (-G8 - G8 + H7 + H7) / 4
        const double g1 = first_order_flux<1>(a, Uold, z, zy)[7], g2 = first_order_flux<1>(a, Uold, zz, zyz)[7];
        const double h1 = first_order_flux<2>(a, Uold, z, zz)[6], h2 = first_order_flux<2>(a, Uold, zy, zyz)[6];
        E[z] = 0.25 * (-g1 - g2 + h1 + h2);
    }
}

// MHD: Eq. 8 again from the face field of step n on the faces with an edge next to a marked zone (the
// others keep the step's value, which the same arithmetic gives).  Zone z owns its faces i-1/2, j-1/2,
// k-1/2 (as in zone_ct), whose edges are stored one zone lower along the face's normal; a face's four
// edges touch the zones within one of it in the face's plane, on both of its sides.
__global__ void __launch_bounds__(128) k_pos_ct(StepArgs a, double* __restrict__ Bf, const double* __restrict__ Bold,
                                                const unsigned char* __restrict__ mark, double c_host,
                                                int use_dt_dev) {
    const Grid& g = a.grid;
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= g.n) return;
    int i, j, k;
    zone_ijk(g, z, i, j, k);
    bool near[3] = {false, false, false};          // x, y, z faces of zone z
#pragma unroll
    for (int dk = -1; dk <= 1; ++dk)
#pragma unroll
        for (int dj = -1; dj <= 1; ++dj)
#pragma unroll
            for (int di = -1; di <= 1; ++di) {
                if (!mark[nbr(g, i, j, k, di, dj, dk)]) continue;
                // the face i-1/2 lies between x-offsets -1 and 0; its edges reach one zone along y and z
                near[0] |= di <= 0;
                near[1] |= dj <= 0;
                near[2] |= dk <= 0;
            }
    if (!(near[0] || near[1] || near[2])) return;
    const double* E = (const double*)a.E;
    const long long N = g.n;
    auto Ex = [&](int di, int dj, int dk) { return E[nbr(g, i, j, k, di, dj, dk)]; };
    auto Ey = [&](int di, int dj, int dk) { return E[N + nbr(g, i, j, k, di, dj, dk)]; };
    auto Ez = [&](int di, int dj, int dk) { return E[2 * N + nbr(g, i, j, k, di, dj, dk)]; };
    const double dt = use_dt_dev ? c_host * (*a.dt_dev) : c_host;
    const double idx = a.idx[0], idy = a.idx[1], idz = a.idx[2];
    if (near[0]) Bf[z] = Bold[z] - dt * ((Ez(-1, 0, 0) - Ez(-1, -1, 0)) * idy - (Ey(-1, 0, 0) - Ey(-1, 0, -1)) * idz);
    if (near[1])
        Bf[N + z] = Bold[N + z] - dt * ((Ex(0, -1, 0) - Ex(0, -1, -1)) * idz - (Ez(0, -1, 0) - Ez(-1, -1, 0)) * idx);
    if (near[2])
        Bf[2 * N + z] =
            Bold[2 * N + z] - dt * ((Ey(0, 0, -1) - Ey(-1, 0, -1)) * idx - (Ex(0, 0, -1) - Ex(0, -1, -1)) * idy);
}

// After the passes (the update deferred its own check to here): a zone value that is not finite raises
// FLAG_NONFINITE, and so does, for MHD, a face field value that is not finite: the fallback replaces only
// hydrodynamic face fluxes, so a non-finite edge field written by constrained transport survives its
// passes.  A zone left finite but non-physical (rho <= 0 or P <= 0 after the third pass) raises
// FLAG_UNPHYSICAL, so the step itself reports what the fallback could not mend.
template <int NV>
__global__ void __launch_bounds__(256) k_pos_check(Grid g, const double* __restrict__ U, const double* __restrict__ Bf,
                                                   double gm1, unsigned* flag) {
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= g.n) return;
    bool bad = false;
#pragma unroll
    for (int v = 0; v < 5; ++v) bad |= !isfinite(U[v * g.n + z]);
    if constexpr (NV == 8) {
#pragma unroll
        for (int c = 0; c < 3; ++c) bad |= !isfinite(Bf[c * g.n + z]);
    }
    if (bad)
        raise_flag(flag, FLAG_NONFINITE);
    else if (unphysical<NV>(g, U, Bf, z, gm1))
        raise_flag(flag, FLAG_UNPHYSICAL);
}

}  // namespace

int launch_positivity_fallback(const StepArgs& a, double* U, const double* Uold, const double* Bold,
                               unsigned char* mark, double c_host, bool use_dt_dev, cudaStream_t st) {
    const long long N = a.grid.n;
    if (N <= 0) return 0;
    cudaMemsetAsync(mark, 0, (size_t)N, st);
    const unsigned b256 = (unsigned)((N + 255) / 256), b128 = (unsigned)((N + 127) / 128);
    int n = 0;
    for (int pass = 0; pass < 3; ++pass) {
        if (a.mhd) {
            k_pos_mark<8><<<b256, 256, 0, st>>>(a.grid, U, a.Bface, a.gm1, mark);
            k_pos_faces<8><<<b128, 128, 0, st>>>(a, Uold, mark);
        } else {
            k_pos_mark<5><<<b256, 256, 0, st>>>(a.grid, U, nullptr, a.gm1, mark);
            k_pos_faces<5><<<b128, 128, 0, st>>>(a, Uold, mark);
        }
        k_pos_update<<<b128, 128, 0, st>>>(a, U, Uold, mark, c_host, use_dt_dev ? 1 : 0);
        n += 3;
        if (a.mhd && Bold) {        // first-order edge fields around the marks, Eq. 8 again from step n
            k_pos_emf<<<b128, 128, 0, st>>>(a, Uold, mark);
            k_pos_ct<<<b128, 128, 0, st>>>(a, const_cast<double*>(a.Bface), Bold, mark, c_host, use_dt_dev ? 1 : 0);
            n += 2;
        }
    }
    if (a.mhd)
        k_pos_check<8><<<b256, 256, 0, st>>>(a.grid, U, a.Bface, a.gm1, a.flag);
    else
        k_pos_check<5><<<b256, 256, 0, st>>>(a.grid, U, nullptr, a.gm1, a.flag);
    return n + 1;
}

}  // namespace ader
