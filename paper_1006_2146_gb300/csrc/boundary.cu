// Ghost zones of the non-periodic box faces (Euler): the padded state the step runs on, and the copy
// of its interior back.  The paper's tests with walls and open sides (Sec. VIII) state no boundary
// treatment; the reading is the usual ghost-zone one.  OUTFLOW copies the nearest interior zone (zero
// gradient); REFLECTIVE copies the mirror-image interior zone (ghost -1 - k <- zone k, nx + k <- nx - 1 - k)
// with the momentum normal to the face negated.  The periodic step on the padded state (G ghost zones
// across every non-periodic face, G at least a step's reach) leaves the interior as the boundaries give
// it.
#include "kernels.cuh"

namespace ader {

struct BoxBC {
    int bc[6];          // x-, x+, y-, y+, z-, z+: 0 periodic, 1 outflow, 2 reflective
    int g[3];           // ghost zones on each side of each axis (0 on a periodic axis)
};

// source index along one axis of padded index ip, and whether the ghost is a mirror image
ADER_DEV int bc_source(int ip, int g, int n, int lo, int hi, bool& flip) {
    const int i = ip - g;
    if (i < 0) {
        if (lo == 1) return 0;
        flip = true;
        return -1 - i;
    }
    if (i >= n) {
        if (hi == 1) return n - 1;
        flip = true;
        return 2 * n - 1 - i;
    }
    return i;
}

__global__ void __launch_bounds__(256) k_fill_ghosts(Grid g, Grid gp, BoxBC b, const double* __restrict__ U,
                                                     double* __restrict__ Up) {
    const long long zp = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (zp >= gp.n) return;
    int ip, jp, kp;
    zone_ijk(gp, zp, ip, jp, kp);
    bool fx = false, fy = false, fz = false;
    const int i = bc_source(ip, b.g[0], g.nx, b.bc[0], b.bc[1], fx);
    const int j = bc_source(jp, b.g[1], g.ny, b.bc[2], b.bc[3], fy);
    const int k = bc_source(kp, b.g[2], g.nz, b.bc[4], b.bc[5], fz);
    const long long z = ((long long)k * g.ny + j) * g.nx + i;
    Up[zp] = U[z];
    Up[gp.n + zp] = fx ? -U[g.n + z] : U[g.n + z];
    Up[2 * gp.n + zp] = fy ? -U[2 * g.n + z] : U[2 * g.n + z];
    Up[3 * gp.n + zp] = fz ? -U[3 * g.n + z] : U[3 * g.n + z];
    Up[4 * gp.n + zp] = U[4 * g.n + z];
}

__global__ void __launch_bounds__(256) k_copy_interior(Grid g, Grid gp, BoxBC b, const double* __restrict__ Up,
                                                       double* __restrict__ U) {
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= g.n) return;
    int i, j, k;
    zone_ijk(g, z, i, j, k);
    const long long zp = ((long long)(k + b.g[2]) * gp.ny + (j + b.g[1])) * gp.nx + (i + b.g[0]);
#pragma unroll
    for (int v = 0; v < 5; ++v) U[v * g.n + z] = Up[v * gp.n + zp];
}

int launch_fill_ghosts(const Grid& g, const Grid& gp, const int bc[6], const int gh[3], const double* U, double* Up,
                       cudaStream_t st) {
    BoxBC b;
    for (int s = 0; s < 6; ++s) b.bc[s] = bc[s];
    for (int d = 0; d < 3; ++d) b.g[d] = gh[d];
    k_fill_ghosts<<<(unsigned)((gp.n + 255) / 256), 256, 0, st>>>(g, gp, b, U, Up);
    return 1;
}

int launch_copy_interior(const Grid& g, const Grid& gp, const int gh[3], const double* Up, double* U, cudaStream_t st) {
    BoxBC b{};
    for (int d = 0; d < 3; ++d) b.g[d] = gh[d];
    k_copy_interior<<<(unsigned)((g.n + 255) / 256), 256, 0, st>>>(g, gp, b, Up, U);
    return 1;
}

}  // namespace ader
