// Space-time mode numbering (Eqs. 14-16) and the mode permutations that let
// the paper's x-face formulas (Sec. V, App. D) serve the y- and z-faces and
// the lower faces.
//
// Mode k (1-based) of order M is P_a(xi) P_b(eta) P_c(zeta) tau^d, stored as
// the exponent tuple {a, b, c, d}.  A face with normal direction D is mapped
// onto the x-frame (normal, t1, t2) with t1 < t2 the two other directions in
// increasing order; the lower face (S = -1) additionally reflects the normal
// coordinate, which multiplies mode k by (-1)^(normal exponent).
#pragma once
#include <utility>

#include "common.cuh"

namespace ader {

struct Exp4 { int a, b, c, d; };

// Eq. 14
constexpr Exp4 MODES2[6] = {{0, 0, 0, 0}, {0, 0, 0, 0}, {1, 0, 0, 0}, {0, 1, 0, 0}, {0, 0, 1, 0}, {0, 0, 0, 1}};
// Eq. 15
constexpr Exp4 MODES3[16] = {{0, 0, 0, 0},
                             {0, 0, 0, 0}, {1, 0, 0, 0}, {0, 1, 0, 0}, {0, 0, 1, 0}, {2, 0, 0, 0},
                             {0, 2, 0, 0}, {0, 0, 2, 0}, {1, 1, 0, 0}, {0, 1, 1, 0}, {1, 0, 1, 0},
                             {0, 0, 0, 1}, {0, 0, 0, 2}, {1, 0, 0, 1}, {0, 1, 0, 1}, {0, 0, 1, 1}};
// Eq. 16
constexpr Exp4 MODES4[36] = {{0, 0, 0, 0},
                             {0, 0, 0, 0}, {1, 0, 0, 0}, {0, 1, 0, 0}, {0, 0, 1, 0}, {2, 0, 0, 0},
                             {0, 2, 0, 0}, {0, 0, 2, 0}, {1, 1, 0, 0}, {0, 1, 1, 0}, {1, 0, 1, 0},
                             {3, 0, 0, 0}, {0, 3, 0, 0}, {0, 0, 3, 0}, {2, 1, 0, 0}, {2, 0, 1, 0},
                             {1, 2, 0, 0}, {0, 2, 1, 0}, {1, 0, 2, 0}, {0, 1, 2, 0}, {1, 1, 1, 0},
                             {0, 0, 0, 1}, {0, 0, 0, 2}, {0, 0, 0, 3}, {1, 0, 0, 1}, {0, 1, 0, 1},
                             {0, 0, 1, 1}, {1, 0, 0, 2}, {0, 1, 0, 2}, {0, 0, 1, 2}, {2, 0, 0, 1},
                             {0, 2, 0, 1}, {0, 0, 2, 1}, {1, 1, 0, 1}, {0, 1, 1, 1}, {1, 0, 1, 1}};

template <int ORDER> struct ModeCount;
template <> struct ModeCount<2> { static constexpr int LS = 4, L = 5; };
template <> struct ModeCount<3> { static constexpr int LS = 10, L = 15; };
template <> struct ModeCount<4> { static constexpr int LS = 20, L = 35; };

template <int ORDER>
constexpr Exp4 mode_exp(int k) {
    return ORDER == 2 ? MODES2[k] : (ORDER == 3 ? MODES3[k] : MODES4[k]);
}

template <int ORDER>
constexpr int find_mode(int a, int b, int c, int d) {
    for (int k = 1; k <= ModeCount<ORDER>::L; ++k) {
        const Exp4 e = mode_exp<ORDER>(k);
        if (e.a == a && e.b == b && e.c == c && e.d == d) return k;
    }
    return 0;
}

// index, in the actual zone frame, of x-frame mode k for a face of normal D
template <int ORDER, int D>
constexpr int face_perm(int k) {
    const Exp4 e = mode_exp<ORDER>(k);     // e.a = normal, e.b = t1, e.c = t2
    return D == 0 ? find_mode<ORDER>(e.a, e.b, e.c, e.d)
                  : (D == 1 ? find_mode<ORDER>(e.b, e.a, e.c, e.d) : find_mode<ORDER>(e.b, e.c, e.a, e.d));
}

template <int ORDER, int S>
constexpr int face_sign(int k) {
    return (S < 0 && (mode_exp<ORDER>(k).a & 1)) ? -1 : 1;
}

// p[k] = sign * m[perm(k)]: the zone's modes seen in the x-frame of face (D, S).
// The permutation is resolved at compile time (one statement per mode).
template <int ORDER, int D, int S, int K, int NV, class R>
ADER_DEV void to_face_frame_one(const Vec<NV, R>* m, Vec<NV, R>* p) {
    constexpr int src = face_perm<ORDER, D>(K);
    constexpr int sg = face_sign<ORDER, S>(K);
    static_assert(src >= 1, "mode permutation must be complete");
    p[K] = sg < 0 ? -m[src] : m[src];
}

template <int ORDER, int D, int S, int NV, class R, int... K>
ADER_DEV void to_face_frame_seq(const Vec<NV, R>* m, Vec<NV, R>* p, std::integer_sequence<int, K...>) {
    (to_face_frame_one<ORDER, D, S, K + 1>(m, p), ...);
}

template <int ORDER, int D, int S, int NV, class R>
ADER_DEV void to_face_frame(const Vec<NV, R>* m, Vec<NV, R>* p) {
    to_face_frame_seq<ORDER, D, S>(m, p, std::make_integer_sequence<int, ModeCount<ORDER>::L>{});
}

}  // namespace ader
