// Host tool: exact floating-point operation counts per zone of each kernel.
//
// The kernels' per-zone bodies are templates on the scalar type; this tool
// instantiates them with an op-counting scalar and runs them on the host over
// a small periodic grid.  Counted: add/sub, mul, div, sqrt (one FLOP each;
// an FMA is its mul + add, i.e. two).  min/max/abs/compare are counted
// separately and not included in the FLOP total.  The FP64 accumulation of
// the stored face-flux differences in the update kernel (3 per variable per
// direction, then base + c acc) is added explicitly.
//
// Build and run (host tool; the device side of the headers needs sm_103a):
//   nvcc -O0 -Xcompiler -O0 -std=c++17 --expt-relaxed-constexpr -gencode arch=compute_103a,code=sm_103a \
//        flopcount.cu -o flopcount && ./flopcount
#include <cmath>
#include <cstdio>
#include <vector>

struct Cnt;
static long long g_add = 0, g_mul = 0, g_div = 0, g_sqrt = 0, g_cmp = 0;

struct Cnt {
    double v;
    Cnt() : v(0) {}
    Cnt(double x) : v(x) {}
    explicit operator double() const { return v; }
};
inline Cnt operator+(Cnt a, Cnt b) { ++g_add; return Cnt(a.v + b.v); }
inline Cnt operator-(Cnt a, Cnt b) { ++g_add; return Cnt(a.v - b.v); }
inline Cnt operator*(Cnt a, Cnt b) { ++g_mul; return Cnt(a.v * b.v); }
inline Cnt operator/(Cnt a, Cnt b) { ++g_div; return Cnt(a.v / b.v); }
inline Cnt operator-(Cnt a) { return Cnt(-a.v); }
inline Cnt& operator+=(Cnt& a, Cnt b) { a = a + b; return a; }
inline Cnt& operator-=(Cnt& a, Cnt b) { a = a - b; return a; }
inline bool operator>(Cnt a, Cnt b) { ++g_cmp; return a.v > b.v; }
inline bool operator<(Cnt a, Cnt b) { ++g_cmp; return a.v < b.v; }
inline Cnt sqrt(Cnt a) { ++g_sqrt; return Cnt(std::sqrt(a.v)); }
inline Cnt fmin(Cnt a, Cnt b) { ++g_cmp; return Cnt(std::fmin(a.v, b.v)); }
inline Cnt fmax(Cnt a, Cnt b) { ++g_cmp; return Cnt(std::fmax(a.v, b.v)); }
inline Cnt fabs(Cnt a) { ++g_cmp; return Cnt(std::fabs(a.v)); }
inline Cnt fma(Cnt a, Cnt b, Cnt c) { ++g_mul; ++g_add; return Cnt(std::fma(a.v, b.v, c.v)); }

#include "../weno.cuh"
#include "../step_inst.cuh"

using namespace ader;

static long long flops() { return g_add + g_mul + g_div + g_sqrt; }
static void reset() { g_add = g_mul = g_div = g_sqrt = g_cmp = 0; }

int main() {
    const int n = 6;
    Grid g{n, n, n, (long long)n * n * n};
    const long long N = g.n;
    std::vector<double> U(5 * N);
    for (long long z = 0; z < N; ++z) {
        const double s = 0.1 * std::sin(0.7 * z);
        U[z] = 1.0 + s;
        U[N + z] = 0.3 + s;
        U[2 * N + z] = -0.2 + 0.5 * s;
        U[3 * N + z] = 0.1 - s;
        U[4 * N + z] = 2.5 + s;
    }
    std::printf("{\n");
    for (int order = 2; order <= 4; ++order) {
        std::vector<Cnt> S1(N * 45), S2(N * 50), S3(N * 90);
        StepArgs a{};
        a.grid = g;
        a.order = order;
        a.n_iter = order - 1;
        a.gamma = 1.4;
        a.dx[0] = a.dx[1] = a.dx[2] = 1.0 / n;
        finish_args(a);
        a.dt = 0.01;
        a.S1 = S1.data();
        a.S2 = S2.data();
        a.S3 = S3.data();
        unsigned flag = 0;
        a.flag = &flag;
        reset();
        for (long long z = 0; z < N; ++z) {
            if (order == 2) zone_weno1d<2, 5, Cnt>(g, U.data(), nullptr, S1.data(), z);
            if (order == 3) zone_weno1d<3, 5, Cnt>(g, U.data(), nullptr, S1.data(), z);
            if (order == 4) zone_weno1d<4, 5, Cnt>(g, U.data(), nullptr, S1.data(), z);
        }
        if (order >= 3)
            for (long long z = 0; z < N; ++z) {
                if (order == 3) zone_cross1<3, 5, Cnt>(g, S1.data(), S2.data(), z);
                else zone_cross1<4, 5, Cnt>(g, S1.data(), S2.data(), z);
            }
        if (order == 4)
            for (long long z = 0; z < N; ++z) zone_cross2<5, Cnt>(g, S2.data(), z);
        const double recon = (double)flops() / N;
        std::printf("  \"order%d\": {\"weno_reconstruction\": %.1f", order, recon);
        for (int form = 0; form < 2; ++form) {
            reset();
            for (long long z = 0; z < N; ++z) {
                if (order == 2) form ? zone_predict_faces<2, 1, 5, Cnt>(a, U.data(), z) : zone_predict_faces<2, 0, 5, Cnt>(a, U.data(), z);
                if (order == 3) form ? zone_predict_faces<3, 1, 5, Cnt>(a, U.data(), z) : zone_predict_faces<3, 0, 5, Cnt>(a, U.data(), z);
                if (order == 4) form ? zone_predict_faces<4, 1, 5, Cnt>(a, U.data(), z) : zone_predict_faces<4, 0, 5, Cnt>(a, U.data(), z);
            }
            std::printf(", \"predictor_faces_%s\": %.1f", form ? "nodal" : "modal", (double)flops() / N);
        }
        // spatial-only face data (the SSP-RK operator)
        a.n_iter = 0;
        reset();
        for (long long z = 0; z < N; ++z) {
            if (order == 2) zone_predict_faces<2, 0, 5, Cnt>(a, U.data(), z);
            if (order == 3) zone_predict_faces<3, 0, 5, Cnt>(a, U.data(), z);
            if (order == 4) zone_predict_faces<4, 0, 5, Cnt>(a, U.data(), z);
        }
        std::printf(", \"faces_spatial_only\": %.1f", (double)flops() / N);
        std::vector<double> out(5 * N);
        for (int sol = 0; sol < 2; ++sol) {
            reset();
            // FP64: each face solved once, then the update from the stored fluxes
            for (long long z = 0; z < N; ++z) {
                if (sol == 0) zone_face_fluxes<0, 5, Cnt>(a, z);
                else zone_face_fluxes<1, 5, Cnt>(a, z);
            }
            for (long long z = 0; z < N; ++z) zone_flux_update_stored<Cnt>(a, out.data(), U.data(), 0.01, 0, z);
            // FP64 accumulation: per direction and variable one subtract, one multiply, one subtract; then base + c*acc
            const double acc = 3 * 5 * 3 + 5 * 2;
            std::printf(", \"riemann_update_%s\": %.1f", sol ? "linearized" : "hll", (double)flops() / N + acc);
            // FP32 bulk: each zone solves both faces of each direction (one fused pass)
            reset();
            for (long long z = 0; z < N; ++z) {
                if (sol == 0) zone_flux_update<0, 5, Cnt>(a, out.data(), U.data(), 0.01, 0, z);
                else zone_flux_update<1, 5, Cnt>(a, out.data(), U.data(), 0.01, 0, z);
            }
            std::printf(", \"riemann_update_fused_%s\": %.1f", sol ? "linearized" : "hll", (double)flops() / N + acc);
        }
        std::printf("}%s\n", order < 4 ? "," : "");
    }
    std::printf("}\n");
    return 0;
}
