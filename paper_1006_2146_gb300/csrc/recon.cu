// Zone-centred WENO reconstruction to Hermite modes (Sec. II.1, Eqs. 10-12).
//
// The paper defers the zone-centred scheme to its ref. [11]; this file
// implements the reading stated in the library's design notes:
//   * 1-D, per direction: order 3 (and 2) blends the 3-zone stencils
//     {i-2..i}, {i-1..i+1}, {i..i+2} with linear weights (1, 10, 1)/12; order 4
//     blends the 4-zone stencils {i-3..i} .. {i..i+3} with (1, 10, 10, 1)/22.
//     Each candidate is the polynomial a + b P1 + c P2 (+ d P3) whose zone
//     averages match the stencil (cell average of P1, P2, P3 over zone k is
//     k, k^2, k^3 + k/10).  Order 2 keeps only b.
//   * smoothness IS = b^2 + 13 c^2 / 3 (Eq. 24 form) or
//     (b + d/10)^2 + 13 c^2 / 3 + 781 d^2 / 20 (Eq. 29 form);
//     weights gamma_s / (1e-12 + IS_s)^2, normalised.
//   * cross moments: WENO slope S_e (order-3 candidate set, b kept) of a
//     moment field in a transverse direction, symmetrised:
//     w8 = (S_y w2 + S_x w3)/2, w9 = (S_z w3 + S_y w4)/2, w10 = (S_z w2 + S_x w4)/2,
//     w14 = S_y w5, w15 = S_z w5, w16 = S_x w6, w17 = S_z w6, w18 = S_x w7,
//     w19 = S_y w7, w20 = (S_z w8 + S_x w9 + S_y w10)/3.
//
// Scratch layouts (N = nx*ny*nz zones, NV = 5 variables):
//   S1[((r*3 + d)*NV + v)*N + zone]  1-D moment r (0: P1, 1: P2, 2: P3) along d
//   S2[(c*NV + v)*N + zone]          cross moment c: w8 w9 w10 w14 w15 w16 w17 w18 w19 w20
#include "common.cuh"
#include "kernels.cuh"
#include "weno.cuh"

namespace ader {

// ---------------------------------------------------------------- kernels (one thread per zone)
template <int ORDER, class R>
__global__ void __launch_bounds__(128) k_face_b(Grid g, const double* __restrict__ Bf, R* __restrict__ ZB,
                                                R* __restrict__ S1) {
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (z < g.n) zone_face_b<ORDER, R>(g, Bf, ZB, S1, z);
}

template <int ORDER, int NV, class R, class T>
__global__ void __launch_bounds__(128) k_weno1d(Grid g, const T* __restrict__ U, const R* __restrict__ ZB,
                                                R* __restrict__ S1) {
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (z < g.n) zone_weno1d<ORDER, NV>(g, U, ZB, S1, z);
}

// FP32 copy of the state: every value is rounded once per step here instead of
// at each of the 13 stencil points that read it, with integer operations
// (f32_of_f64; GB300 runs its conversion instruction on the scarce FP64 units).
// Pairs of values per thread, two pairs per pass; an odd last value is taken by
// the first thread.
__global__ void __launch_bounds__(256) k_to_f32(float* __restrict__ out, const double* __restrict__ U, long long count) {
    const long long n2 = count / 2;
    const double2* in = reinterpret_cast<const double2*>(U);
    float2* o = reinterpret_cast<float2*>(out);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += 2 * stride) {
        const double2 v = in[i];
        const bool two = i + stride < n2;
        const double2 w = two ? in[i + stride] : v;
        o[i] = make_float2(f32_of_f64(v.x), f32_of_f64(v.y));
        if (two) o[i + stride] = make_float2(f32_of_f64(w.x), f32_of_f64(w.y));
    }
    if ((count & 1) && blockIdx.x == 0 && threadIdx.x == 0) out[count - 1] = f32_of_f64(U[count - 1]);
}

int launch_to_f32(float* out, const double* U, long long count, cudaStream_t st) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long want = (count / 2 + 255) / 256;
    const unsigned blocks = (unsigned)(want < (long long)sms * 16 ? (want > 0 ? want : 1) : (long long)sms * 16);
    k_to_f32<<<blocks, 256, 0, st>>>(out, U, count);
    return 1;
}

template <int ORDER, int NV, class R>
__global__ void __launch_bounds__(128) k_cross1(Grid g, const R* __restrict__ S1, R* __restrict__ S2) {
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (z < g.n) zone_cross1<ORDER, NV>(g, S1, S2, z);
}

// Third-order cross moments in FP32 from shared-memory tiles (2.5-D
// blocking).  A block of CT_X x CT_Y threads owns a tile of the x-y plane and
// marches through CT_Z planes of z (4 more planes of the z window are read per chunk).  Each thread keeps w2 and w3 of its column
// at z-2..z+2 in registers (for the z slopes); the plane z of w2 (with y
// halos), w3 (x halos) and w4 (both) sits in shared memory for the x and y
// slopes.  Every moment is read about once per zone and plane instead of once
// per neighbour stencil that uses it; the arithmetic is zone_cross1's.
// Requires nx % CT_X == 0 and ny % CT_Y == 0 (other grids use k_cross1).
constexpr int CT_X = 32, CT_Y = 8, CT_Z = 8;    // 8-plane chunks: enough blocks to fill the SMs from 128^3 up

template <int NV>
__global__ void __launch_bounds__(CT_X * CT_Y) k_cross1_tiled(Grid g, const float* __restrict__ S1,
                                                              float* __restrict__ S2) {
    __shared__ float s2[CT_Y + 4][CT_X];          // w2 with two rows of y halo on each side
    __shared__ float s3[CT_Y][CT_X + 4];          // w3 with two columns of x halo
    __shared__ float s4[CT_Y + 4][CT_X + 4];      // w4 with both
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tiles_x = g.nx / CT_X;
    const int i = (int)(blockIdx.x % tiles_x) * CT_X + tx, j = (int)(blockIdx.x / tiles_x) * CT_Y + ty;
    const int k0 = (int)blockIdx.y * CT_Z, k1 = min(k0 + CT_Z, g.nz);
    const long long N = g.n;
    // periodic offsets, once per thread: the column (i, j), its y and x halos, and the z planes
    const long long nxy = (long long)g.nx * g.ny;
    const long long xy = (long long)j * g.nx + i;
    const long long xy_jm = (long long)wrap(j - 2, g.ny) * g.nx + i, xy_jp = (long long)wrap(j + 2, g.ny) * g.nx + i;
    const long long xy_im = (long long)j * g.nx + wrap(i - 2, g.nx), xy_ip = (long long)j * g.nx + wrap(i + 2, g.nx);
    auto plane = [&](int kk) -> long long { return (long long)wrap(kk, g.nz) * nxy; };
    for (int v = 0; v < NV; ++v) {
        const float* w2 = S1 + ((0 * 3 + 0) * NV + v) * N;
        const float* w3 = S1 + ((0 * 3 + 1) * NV + v) * N;
        const float* w4 = S1 + ((0 * 3 + 2) * NV + v) * N;
        float c2[5], c3[5];                        // the column at z - 2 .. z + 2
#pragma unroll
        for (int o = -2; o <= 1; ++o) {
            const long long p = plane(k0 + o) + xy;
            c2[o + 3] = w2[p];
            c3[o + 3] = w3[p];
        }
        for (int k = k0; k < k1; ++k) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                c2[q] = c2[q + 1];
                c3[q] = c3[q + 1];
            }
            const long long p2 = plane(k + 2) + xy;
            c2[4] = w2[p2];
            c3[4] = w3[p2];
            // the plane k (k < nz) with its halos
            const long long pk = (long long)k * nxy;
            s2[ty + 2][tx] = c2[2];
            s3[ty][tx + 2] = c3[2];
            s4[ty + 2][tx + 2] = w4[pk + xy];
            if (ty < 2) {
                s2[ty][tx] = w2[pk + xy_jm];
                s4[ty][tx + 2] = w4[pk + xy_jm];
            }
            if (ty >= CT_Y - 2) {
                s2[ty + 4][tx] = w2[pk + xy_jp];
                s4[ty + 4][tx + 2] = w4[pk + xy_jp];
            }
            if (tx < 2) {
                s3[ty][tx] = w3[pk + xy_im];
                s4[ty + 2][tx] = w4[pk + xy_im];
            }
            if (tx >= CT_X - 2) {
                s3[ty][tx + 4] = w3[pk + xy_ip];
                s4[ty + 2][tx + 4] = w4[pk + xy_ip];
            }
            __syncthreads();
            // the six slopes in three packed pairs (weno3_x2): (S_y w2, S_x w3), (S_z w3, S_y w4),
            // (S_z w2, S_x w4) -- each pair is also the pair of terms of one cross moment
            float2 a[5], r0, r1, r2, unused;
#pragma unroll
            for (int o = 0; o < 5; ++o) a[o] = make_float2(s2[ty + o][tx], s3[ty][tx + o]);
            weno3_x2<false>(a, r0, unused);
#pragma unroll
            for (int o = 0; o < 5; ++o) a[o] = make_float2(c3[o], s4[ty + o][tx + 2]);
            weno3_x2<false>(a, r1, unused);
#pragma unroll
            for (int o = 0; o < 5; ++o) a[o] = make_float2(c2[o], s4[ty + 2][tx + o]);
            weno3_x2<false>(a, r2, unused);
            const long long z = pk + xy;
            S2[(0 * NV + v) * N + z] = 0.5f * (r0.x + r0.y);
            S2[(1 * NV + v) * N + z] = 0.5f * (r1.x + r1.y);
            S2[(2 * NV + v) * N + z] = 0.5f * (r2.x + r2.y);
            __syncthreads();
        }
    }
}

template <int NV>
static bool launch_cross1_tiled(const Grid& g, const float* S1, float* S2, cudaStream_t st) {
    if (g.nx % CT_X != 0 || g.ny % CT_Y != 0) return false;
    const dim3 grid((unsigned)((g.nx / CT_X) * (g.ny / CT_Y)), (unsigned)((g.nz + CT_Z - 1) / CT_Z));
    k_cross1_tiled<NV><<<grid, dim3(CT_X, CT_Y), 0, st>>>(g, S1, S2);
    return true;
}

// FP64 third-order cross moments from shared-memory tiles, each slope's per-position WENO terms (d, E of
// weno3_terms) computed once per position.  The tile and the z march are k_cross1_tiled's (CT_X x CT_Y
// threads, CT_Z planes per block); the planes of w2, w3, w4 with their halos go to shared memory, and
// from them the terms of the x slopes (w3, w4: positions i0-1 .. i0+33 for d, i0-1 .. i0+32 for E) and
// of the y slopes (w2, w4: rows j0-1 .. j0+9 and j0-1 .. j0+8); each thread keeps the z terms of its
// column (w2, w3) in registers and slides them up one plane at a time.  A zone's slope then takes four
// d and three E from there: about 27 FP64 operations instead of 39.  Same bits as zone_cross1.
// Requires nx % CT_X == 0 and ny % CT_Y == 0 (other grids use k_cross1).
template <int NV>
__global__ void __launch_bounds__(CT_X * CT_Y) k_cross1_tiled64(Grid g, const double* __restrict__ S1,
                                                                double* __restrict__ S2) {
    __shared__ double s2[CT_Y + 4][CT_X];          // w2 with two rows of y halo on each side
    __shared__ double s3[CT_Y][CT_X + 4];          // w3 with two columns of x halo
    __shared__ double s4[CT_Y + 4][CT_X + 4];      // w4 with both
    __shared__ double dx3[CT_Y][CT_X + 3], dx4[CT_Y][CT_X + 3];    // d along x at i0 - 1 + c
    __shared__ double ex3[CT_Y][CT_X + 2], ex4[CT_Y][CT_X + 2];    // E along x at i0 - 1 + c
    __shared__ double dy2[CT_Y + 3][CT_X], dy4[CT_Y + 3][CT_X];    // d along y at j0 - 1 + r
    __shared__ double ey2[CT_Y + 2][CT_X], ey4[CT_Y + 2][CT_X];    // E along y at j0 - 1 + r
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tiles_x = g.nx / CT_X;
    const int i = (int)(blockIdx.x % tiles_x) * CT_X + tx, j = (int)(blockIdx.x / tiles_x) * CT_Y + ty;
    const int k0 = (int)blockIdx.y * CT_Z, k1 = min(k0 + CT_Z, g.nz);
    const long long N = g.n;
    const long long nxy = (long long)g.nx * g.ny;
    const long long xy = (long long)j * g.nx + i;
    const long long xy_jm = (long long)wrap(j - 2, g.ny) * g.nx + i, xy_jp = (long long)wrap(j + 2, g.ny) * g.nx + i;
    const long long xy_im = (long long)j * g.nx + wrap(i - 2, g.nx), xy_ip = (long long)j * g.nx + wrap(i + 2, g.nx);
    auto plane = [&](int kk) -> long long { return (long long)wrap(kk, g.nz) * nxy; };
    // the halo entries of the term arrays: along x, threads tx = 0, 1, 2 of each row add the positions -1,
    // 32, 33 (d) and tx = 0, 1 the positions -1, 32 (E); along y, rows ty = 0, 1, 2 and ty = 0, 1 likewise
    const int hx_d = tx == 0 ? 0 : CT_X + tx;          // d index of the extra position (tx < 3): 0, 33, 34
    const int hx_e = tx == 0 ? 0 : CT_X + 1;           // E index of the extra position (tx < 2): 0, 33
    const int hy_d = ty == 0 ? 0 : CT_Y + ty;          // (ty < 3): 0, 9, 10
    const int hy_e = ty == 0 ? 0 : CT_Y + 1;           // (ty < 2): 0, 9
    for (int v = 0; v < NV; ++v) {
        const double* w2 = S1 + ((0 * 3 + 0) * NV + v) * N;
        const double* w3 = S1 + ((0 * 3 + 1) * NV + v) * N;
        const double* w4 = S1 + ((0 * 3 + 2) * NV + v) * N;
        // z terms of the column: c = w at k-2 .. k+2, d at k-1 .. k+2, E at k-1 .. k+1
        double c2[5], c3[5], dz2[4], dz3[4], ez2[3], ez3[3];
#pragma unroll
        for (int o = -2; o <= 2; ++o) {
            const long long p = plane(k0 + o) + xy;
            c2[o + 2] = w2[p];
            c3[o + 2] = w3[p];
        }
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            dz2[s] = rn_sub(c2[s + 1], c2[s]);
            dz3[s] = rn_sub(c3[s + 1], c3[s]);
        }
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            ez2[s] = w3_curv(rn_sub(dz2[s + 1], dz2[s]));
            ez3[s] = w3_curv(rn_sub(dz3[s + 1], dz3[s]));
        }
        for (int k = k0; k < k1; ++k) {
            if (k > k0) {              // slide the column up one plane
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    c2[q] = c2[q + 1];
                    c3[q] = c3[q + 1];
                }
                const long long p2 = plane(k + 2) + xy;
                c2[4] = w2[p2];
                c3[4] = w3[p2];
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    dz2[q] = dz2[q + 1];
                    dz3[q] = dz3[q + 1];
                }
                dz2[3] = rn_sub(c2[4], c2[3]);
                dz3[3] = rn_sub(c3[4], c3[3]);
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    ez2[q] = ez2[q + 1];
                    ez3[q] = ez3[q + 1];
                }
                ez2[2] = w3_curv(rn_sub(dz2[3], dz2[2]));
                ez3[2] = w3_curv(rn_sub(dz3[3], dz3[2]));
            }
            // the plane k with its halos
            const long long pk = (long long)k * nxy;
            s2[ty + 2][tx] = c2[2];
            s3[ty][tx + 2] = c3[2];
            s4[ty + 2][tx + 2] = w4[pk + xy];
            if (ty < 2) {
                s2[ty][tx] = w2[pk + xy_jm];
                s4[ty][tx + 2] = w4[pk + xy_jm];
            }
            if (ty >= CT_Y - 2) {
                s2[ty + 4][tx] = w2[pk + xy_jp];
                s4[ty + 4][tx + 2] = w4[pk + xy_jp];
            }
            if (tx < 2) {
                s3[ty][tx] = w3[pk + xy_im];
                s4[ty + 2][tx] = w4[pk + xy_im];
            }
            if (tx >= CT_X - 2) {
                s3[ty][tx + 4] = w3[pk + xy_ip];
                s4[ty + 2][tx + 4] = w4[pk + xy_ip];
            }
            __syncthreads();
            // d: own position (index + 1), then the halo positions; d at index c is w(c) - w(c - 1) in
            // the shifted columns (x: s[.][c + 1] - s[.][c]; y: s[r + 1][.] - s[r][.])
            dx3[ty][tx + 1] = rn_sub(s3[ty][tx + 2], s3[ty][tx + 1]);
            dx4[ty][tx + 1] = rn_sub(s4[ty + 2][tx + 2], s4[ty + 2][tx + 1]);
            dy2[ty + 1][tx] = rn_sub(s2[ty + 2][tx], s2[ty + 1][tx]);
            dy4[ty + 1][tx] = rn_sub(s4[ty + 2][tx + 2], s4[ty + 1][tx + 2]);
            if (tx < 3) {
                dx3[ty][hx_d] = rn_sub(s3[ty][hx_d + 1], s3[ty][hx_d]);
                dx4[ty][hx_d] = rn_sub(s4[ty + 2][hx_d + 1], s4[ty + 2][hx_d]);
            }
            if (ty < 3) {
                dy2[hy_d][tx] = rn_sub(s2[hy_d + 1][tx], s2[hy_d][tx]);
                dy4[hy_d][tx] = rn_sub(s4[hy_d + 1][tx + 2], s4[hy_d][tx + 2]);
            }
            __syncthreads();
            ex3[ty][tx + 1] = w3_curv(rn_sub(dx3[ty][tx + 2], dx3[ty][tx + 1]));
            ex4[ty][tx + 1] = w3_curv(rn_sub(dx4[ty][tx + 2], dx4[ty][tx + 1]));
            ey2[ty + 1][tx] = w3_curv(rn_sub(dy2[ty + 2][tx], dy2[ty + 1][tx]));
            ey4[ty + 1][tx] = w3_curv(rn_sub(dy4[ty + 2][tx], dy4[ty + 1][tx]));
            if (tx < 2) {
                ex3[ty][hx_e] = w3_curv(rn_sub(dx3[ty][hx_e + 1], dx3[ty][hx_e]));
                ex4[ty][hx_e] = w3_curv(rn_sub(dx4[ty][hx_e + 1], dx4[ty][hx_e]));
            }
            if (ty < 2) {
                ey2[hy_e][tx] = w3_curv(rn_sub(dy2[hy_e + 1][tx], dy2[hy_e][tx]));
                ey4[hy_e][tx] = w3_curv(rn_sub(dy4[hy_e + 1][tx], dy4[hy_e][tx]));
            }
            __syncthreads();
            // the six slopes of zone (i, j, k): four d and three E each
            double d[4], E[3], unused;
            double sy2, sx3, sz3, sy4, sz2, sx4;
#pragma unroll
            for (int q = 0; q < 4; ++q) d[q] = dy2[ty + q][tx];
#pragma unroll
            for (int q = 0; q < 3; ++q) E[q] = ey2[ty + q][tx];
            weno3_terms<false, double>(d, E, nullptr, sy2, unused);
#pragma unroll
            for (int q = 0; q < 4; ++q) d[q] = dx3[ty][tx + q];
#pragma unroll
            for (int q = 0; q < 3; ++q) E[q] = ex3[ty][tx + q];
            weno3_terms<false, double>(d, E, nullptr, sx3, unused);
            weno3_terms<false, double>(dz3, ez3, nullptr, sz3, unused);
#pragma unroll
            for (int q = 0; q < 4; ++q) d[q] = dy4[ty + q][tx];
#pragma unroll
            for (int q = 0; q < 3; ++q) E[q] = ey4[ty + q][tx];
            weno3_terms<false, double>(d, E, nullptr, sy4, unused);
            weno3_terms<false, double>(dz2, ez2, nullptr, sz2, unused);
#pragma unroll
            for (int q = 0; q < 4; ++q) d[q] = dx4[ty][tx + q];
#pragma unroll
            for (int q = 0; q < 3; ++q) E[q] = ex4[ty][tx + q];
            weno3_terms<false, double>(d, E, nullptr, sx4, unused);
            const long long z = pk + xy;
            S2[(0 * NV + v) * N + z] = rn_mul(0.5, rn_add(sy2, sx3));
            S2[(1 * NV + v) * N + z] = rn_mul(0.5, rn_add(sz3, sy4));
            S2[(2 * NV + v) * N + z] = rn_mul(0.5, rn_add(sz2, sx4));
        }
        __syncthreads();           // the next variable's first plane overwrites the tiles
    }
}

// FP64 1-D moments at orders 2-3 (w2..w4, and w5..w7 at order 3) in the same tiles: the plane of each
// variable with two zones of halo in x and y in shared memory, from it the per-position terms (d, D2, E)
// along x and y, the z terms in registers per column; each zone then blends from four d, three D2 and
// three E per direction (weno3_terms).  MHD field components (v >= 5) come from the face-B WENO's zone
// means, and their own direction is left to it, as in zone_weno1d.  Same bits as zone_weno1d.
// Requires nx % CT_X == 0 and ny % CT_Y == 0 (other grids use k_weno1d).
template <int ORDER, int NV>
__global__ void __launch_bounds__(CT_X * CT_Y) k_weno1d_tiled64(Grid g, const double* __restrict__ U,
                                                                const double* __restrict__ ZB,
                                                                double* __restrict__ S1) {
    constexpr bool WANT_C = ORDER == 3;
    __shared__ double su[CT_Y + 4][CT_X + 4];                         // the plane, x and y halos of two
    __shared__ double dx[CT_Y][CT_X + 3], cx[CT_Y][CT_X + 2], ex[CT_Y][CT_X + 2];   // at i0 - 1 + c
    __shared__ double dy[CT_Y + 3][CT_X], cy[CT_Y + 2][CT_X], ey[CT_Y + 2][CT_X];   // at j0 - 1 + r
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tiles_x = g.nx / CT_X;
    const int i = (int)(blockIdx.x % tiles_x) * CT_X + tx, j = (int)(blockIdx.x / tiles_x) * CT_Y + ty;
    const int k0 = (int)blockIdx.y * CT_Z, k1 = min(k0 + CT_Z, g.nz);
    const long long N = g.n;
    const long long nxy = (long long)g.nx * g.ny;
    const long long xy = (long long)j * g.nx + i;
    const long long xy_jm = (long long)wrap(j - 2, g.ny) * g.nx + i, xy_jp = (long long)wrap(j + 2, g.ny) * g.nx + i;
    const long long xy_im = (long long)j * g.nx + wrap(i - 2, g.nx), xy_ip = (long long)j * g.nx + wrap(i + 2, g.nx);
    auto plane = [&](int kk) -> long long { return (long long)wrap(kk, g.nz) * nxy; };
    const int hx_d = tx == 0 ? 0 : CT_X + tx;          // halo entries, as in k_cross1_tiled64
    const int hx_e = tx == 0 ? 0 : CT_X + 1;
    const int hy_d = ty == 0 ? 0 : CT_Y + ty;
    const int hy_e = ty == 0 ? 0 : CT_Y + 1;
    for (int v = 0; v < NV; ++v) {
        const double* u = v < 5 ? U + (long long)v * N : ZB + (long long)(v - 5) * N;
        const int own = v >= 5 ? v - 5 : -1;           // an MHD field's own direction: not reconstructed here
        double c[5], dz[4], cz[3], ez[3];
#pragma unroll
        for (int o = -2; o <= 2; ++o) c[o + 2] = u[plane(k0 + o) + xy];
#pragma unroll
        for (int q = 0; q < 4; ++q) dz[q] = rn_sub(c[q + 1], c[q]);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            cz[q] = rn_sub(dz[q + 1], dz[q]);
            ez[q] = w3_curv(cz[q]);
        }
        for (int k = k0; k < k1; ++k) {
            if (k > k0) {
#pragma unroll
                for (int q = 0; q < 4; ++q) c[q] = c[q + 1];
                c[4] = u[plane(k + 2) + xy];
#pragma unroll
                for (int q = 0; q < 3; ++q) dz[q] = dz[q + 1];
                dz[3] = rn_sub(c[4], c[3]);
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    cz[q] = cz[q + 1];
                    ez[q] = ez[q + 1];
                }
                cz[2] = rn_sub(dz[3], dz[2]);
                ez[2] = w3_curv(cz[2]);
            }
            const long long pk = (long long)k * nxy;
            su[ty + 2][tx + 2] = c[2];
            if (ty < 2) su[ty][tx + 2] = u[pk + xy_jm];
            if (ty >= CT_Y - 2) su[ty + 4][tx + 2] = u[pk + xy_jp];
            if (tx < 2) su[ty + 2][tx] = u[pk + xy_im];
            if (tx >= CT_X - 2) su[ty + 2][tx + 4] = u[pk + xy_ip];
            __syncthreads();
            dx[ty][tx + 1] = rn_sub(su[ty + 2][tx + 2], su[ty + 2][tx + 1]);
            dy[ty + 1][tx] = rn_sub(su[ty + 2][tx + 2], su[ty + 1][tx + 2]);
            if (tx < 3) dx[ty][hx_d] = rn_sub(su[ty + 2][hx_d + 1], su[ty + 2][hx_d]);
            if (ty < 3) dy[hy_d][tx] = rn_sub(su[hy_d + 1][tx + 2], su[hy_d][tx + 2]);
            __syncthreads();
            cx[ty][tx + 1] = rn_sub(dx[ty][tx + 2], dx[ty][tx + 1]);
            ex[ty][tx + 1] = w3_curv(cx[ty][tx + 1]);
            cy[ty + 1][tx] = rn_sub(dy[ty + 2][tx], dy[ty + 1][tx]);
            ey[ty + 1][tx] = w3_curv(cy[ty + 1][tx]);
            if (tx < 2) {
                cx[ty][hx_e] = rn_sub(dx[ty][hx_e + 1], dx[ty][hx_e]);
                ex[ty][hx_e] = w3_curv(cx[ty][hx_e]);
            }
            if (ty < 2) {
                cy[hy_e][tx] = rn_sub(dy[hy_e + 1][tx], dy[hy_e][tx]);
                ey[hy_e][tx] = w3_curv(cy[hy_e][tx]);
            }
            __syncthreads();
            const long long z = pk + xy;
            double d[4], D2[3], E[3], b, cc;
            if (own != 0) {
#pragma unroll
                for (int q = 0; q < 4; ++q) d[q] = dx[ty][tx + q];
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    D2[q] = cx[ty][tx + q];
                    E[q] = ex[ty][tx + q];
                }
                weno3_terms<WANT_C, double>(d, E, D2, b, cc);
                S1[((0 * 3 + 0) * NV + v) * N + z] = b;
                if (WANT_C) S1[((1 * 3 + 0) * NV + v) * N + z] = cc;
            }
            if (own != 1) {
#pragma unroll
                for (int q = 0; q < 4; ++q) d[q] = dy[ty + q][tx];
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    D2[q] = cy[ty + q][tx];
                    E[q] = ey[ty + q][tx];
                }
                weno3_terms<WANT_C, double>(d, E, D2, b, cc);
                S1[((0 * 3 + 1) * NV + v) * N + z] = b;
                if (WANT_C) S1[((1 * 3 + 1) * NV + v) * N + z] = cc;
            }
            if (own != 2) {
                weno3_terms<WANT_C, double>(dz, ez, cz, b, cc);
                S1[((0 * 3 + 2) * NV + v) * N + z] = b;
                if (WANT_C) S1[((1 * 3 + 2) * NV + v) * N + z] = cc;
            }
        }
        __syncthreads();
    }
}

template <int ORDER, int NV>
static bool launch_weno1d_tiled64(const Grid& g, const double* U, const double* ZB, double* S1, cudaStream_t st) {
    if (g.nx % CT_X != 0 || g.ny % CT_Y != 0) return false;
    const dim3 grid((unsigned)((g.nx / CT_X) * (g.ny / CT_Y)), (unsigned)((g.nz + CT_Z - 1) / CT_Z));
    k_weno1d_tiled64<ORDER, NV><<<grid, dim3(CT_X, CT_Y), 0, st>>>(g, U, ZB, S1);
    return true;
}

template <int NV>
static bool launch_cross1_tiled64(const Grid& g, const double* S1, double* S2, cudaStream_t st) {
    if (g.nx % CT_X != 0 || g.ny % CT_Y != 0) return false;
    const dim3 grid((unsigned)((g.nx / CT_X) * (g.ny / CT_Y)), (unsigned)((g.nz + CT_Z - 1) / CT_Z));
    k_cross1_tiled64<NV><<<grid, dim3(CT_X, CT_Y), 0, st>>>(g, S1, S2);
    return true;
}

template <int NV, class R>
__global__ void __launch_bounds__(128) k_cross2(Grid g, R* __restrict__ S2) {
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (z < g.n) zone_cross2<NV>(g, S2, z);
}

template <int NV, class R>
static int launch_recon_nv(const StepArgs& a, const double* U, cudaStream_t st) {
    const int T = 128;
    const unsigned blocks = (unsigned)((a.grid.n + T - 1) / T);
    R* S1 = (R*)a.S1;
    R* S2 = (R*)a.S2;
    R* ZB = (R*)a.ZB;
    int n = 0;
    if (NV == 8) {
        switch (a.order) {
            case 2: k_face_b<2, R><<<blocks, T, 0, st>>>(a.grid, a.Bface, ZB, S1); break;
            case 3: k_face_b<3, R><<<blocks, T, 0, st>>>(a.grid, a.Bface, ZB, S1); break;
            default: k_face_b<4, R><<<blocks, T, 0, st>>>(a.grid, a.Bface, ZB, S1); break;
        }
        n = 1;
    }
    // the state in the bulk precision: FP32 steps read a copy rounded once per step
    using In = R;
    const In* Ui;
    if constexpr (sizeof(R) == 4) {
        n += launch_to_f32(const_cast<float*>(a.Uf), U, 5 * a.grid.n, st);
        Ui = a.Uf;
    } else {
        Ui = U;
    }
    // FP64 orders 2-3: the 1-D moments from shared-memory tiles where the grid allows them
    bool tiled1d = false;
    if constexpr (sizeof(R) == 8) {
        if (a.tiled && a.order == 2) tiled1d = launch_weno1d_tiled64<2, NV>(a.grid, Ui, ZB, S1, st);
        if (a.tiled && a.order == 3) tiled1d = launch_weno1d_tiled64<3, NV>(a.grid, Ui, ZB, S1, st);
    }
    switch (a.order) {
        case 2:
            if (!tiled1d) k_weno1d<2, NV, R, In><<<blocks, T, 0, st>>>(a.grid, Ui, ZB, S1);
            n += 1;
            break;
        case 3:
            if (!tiled1d) k_weno1d<3, NV, R, In><<<blocks, T, 0, st>>>(a.grid, Ui, ZB, S1);
            // shared-memory tiles where the grid allows them (and the context has not turned tiles off)
            if constexpr (sizeof(R) == 4) {
                if (!(a.tiled && launch_cross1_tiled<NV>(a.grid, S1, S2, st)))
                    k_cross1<3, NV, R><<<blocks, T, 0, st>>>(a.grid, S1, S2);
            } else {
                if (!(a.tiled && launch_cross1_tiled64<NV>(a.grid, S1, S2, st)))
                    k_cross1<3, NV, R><<<blocks, T, 0, st>>>(a.grid, S1, S2);
            }
            n += 2;
            break;
        default:
            k_weno1d<4, NV, R, In><<<blocks, T, 0, st>>>(a.grid, Ui, ZB, S1);
            k_cross1<4, NV, R><<<blocks, T, 0, st>>>(a.grid, S1, S2);
            k_cross2<NV, R><<<blocks, T, 0, st>>>(a.grid, S2);
            n += 3;
    }
    return n;
}

template <class R>
int launch_recon(const StepArgs& a, const double* U, cudaStream_t st) {
    return a.mhd ? launch_recon_nv<8, R>(a, U, st) : launch_recon_nv<5, R>(a, U, st);
}

template int launch_recon<double>(const StepArgs&, const double*, cudaStream_t);
template int launch_recon<float>(const StepArgs&, const double*, cudaStream_t);

}  // namespace ader
