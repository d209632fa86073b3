// Second order: ADER-CG predictor (modal Sec. IV.1, nodal App. A) and the x+
// face quantities (Sec. V.1, App. D).  Modes m[1..5] (Eq. 14).
#pragma once
#include "common.cuh"
#include "modes.cuh"

namespace ader {
namespace o2 {

template <int NV, class R>
ADER_DEV void finish_o2(Vec<NV, R>* m, const Vec<NV, R>& n5, PredCtl& ctl) {
    const bool conv = positive_arg(ctl.tol);
    const int cap = conv ? ctl.max_iter : ctl.n_iter;
    const R ref = max_abs(m[1]) + R(sizeof(R) == 8 ? 1e-300 : 1e-30);   // never zero in R
    ctl.iters = 0;
    ctl.capped = conv;
    for (int it = 0; it < cap; ++it) {
        const R change = max_abs_diff(n5, m[5]);
        m[5] = n5;
        ++ctl.iters;
        if (conv && change < R(ctl.tol) * ref) {
            ctl.capped = false;
            break;
        }
    }
}


// Eqs. 31-33 and 30 (one iteration, no sources)
// The update uses only tau = 0 fluxes, so one step reaches the fixed point
// (in converged mode a second step confirms it).
template <int NV, class R>
ADER_DEV void predict_modal(Vec<NV, R>* m, R gm1, R cx, R cy, R cz, PredCtl& ctl) {
    const Vec<NV, R> u1 = m[1] + 0.5 * m[2], u2 = m[1] - 0.5 * m[2];
    const Vec<NV, R> u3 = m[1] + 0.5 * m[3], u4 = m[1] - 0.5 * m[3];
    const Vec<NV, R> u5 = m[1] + 0.5 * m[4], u6 = m[1] - 0.5 * m[4];
    const Vec<NV, R> F2 = scale(cx, flux<0>(u1, gm1) - flux<0>(u2, gm1));
    const Vec<NV, R> G3 = scale(cy, flux<1>(u3, gm1) - flux<1>(u4, gm1));
    const Vec<NV, R> H4 = scale(cz, flux<2>(u5, gm1) - flux<2>(u6, gm1));
    const Vec<NV, R> n5 = -(F2 + G3 + H4);
    finish_o2(m, n5, ctl);
}

// Eqs. A.5, A.4 (h term at node 4, the zeta node of Eq. A.1) and A.6
template <int NV, class R>
ADER_DEV void predict_nodal(Vec<NV, R>* m, R gm1, R cx, R cy, R cz, PredCtl& ctl) {
    const Vec<NV, R> u1 = m[1];
    const Vec<NV, R> u2 = m[1] + 0.5 * m[2], u3 = m[1] + 0.5 * m[3], u4 = m[1] + 0.5 * m[4];
    const Prim<NV, R> p1 = primitives(u1, gm1);
    const Vec<NV, R> u5 = u1 - 2.0 * (scale(cx, flux<0>(u2, gm1) - flux_from<0>(u1, p1)) +
                                scale(cy, flux<1>(u3, gm1) - flux_from<1>(u1, p1)) +
                                scale(cz, flux<2>(u4, gm1) - flux_from<2>(u1, p1)));
    finish_o2(m, u5 - u1, ctl);
}

// ---- with a non-stiff source (s = dt S at the nodes of the current iterate)
// The update of u5 now depends on u5 through the source at the tau = 1 node,
// so each iteration recomputes it; sdt receives dt S-bar from the final
// iterate.  `next(m5)` gives the new u5 for the current one.
template <int NV, class R, class Next>
ADER_DEV void iterate_o2(Vec<NV, R>* m, PredCtl& ctl, Next next) {
    const bool conv = positive_arg(ctl.tol);
    const int cap = conv ? ctl.max_iter : ctl.n_iter;
    const R ref = max_abs(m[1]) + R(sizeof(R) == 8 ? 1e-300 : 1e-30);   // never zero in R
    ctl.iters = 0;
    ctl.capped = conv;
    for (int it = 0; it < cap; ++it) {
        const Vec<NV, R> n5 = next(m[5]);
        const R change = max_abs_diff(n5, m[5]);
        m[5] = n5;
        ++ctl.iters;
        if (conv && change < R(ctl.tol) * ref) {
            ctl.capped = false;
            break;
        }
    }
}

// Eqs. 31-34, 30 and 35: s at the seven nodes of Eq. 31 (node 7 = u1 + u5 at tau = 1)
constexpr bool HAS_SOURCE = true;
constexpr bool HAS_SOURCE_MODAL = true;

template <int NV, class R>
ADER_DEV void predict_modal_src(Vec<NV, R>* m, R gm1, R cx, R cy, R cz, PredCtl& ctl, const Src<R>& src,
                                Vec<NV, R>& sdt) {
    const Vec<NV, R> u1 = m[1] + 0.5 * m[2], u2 = m[1] - 0.5 * m[2];
    const Vec<NV, R> u3 = m[1] + 0.5 * m[3], u4 = m[1] - 0.5 * m[3];
    const Vec<NV, R> u5 = m[1] + 0.5 * m[4], u6 = m[1] - 0.5 * m[4];
    const Vec<NV, R> F2 = scale(cx, flux<0>(u1, gm1) - flux<0>(u2, gm1));
    const Vec<NV, R> G3 = scale(cy, flux<1>(u3, gm1) - flux<1>(u4, gm1));
    const Vec<NV, R> H4 = scale(cz, flux<2>(u5, gm1) - flux<2>(u6, gm1));
    const Vec<NV, R> s1 = (source_at(u1, src) + source_at(u2, src) + source_at(u3, src) + source_at(u4, src) +
                           source_at(u5, src) + source_at(u6, src)) / 6.0;          // Eq. 34
    const Vec<NV, R> base = s1 - (F2 + G3 + H4);
    iterate_o2(m, ctl, [&](const Vec<NV, R>& m5) {
        const Vec<NV, R> s5 = source_at(m[1] + m5, src) - s1;                      // Eq. 34
        return base + (2.0 / 3.0) * s5;                                             // Eq. 30
    });
    sdt = s1 + 0.5 * (source_at(m[1] + m[5], src) - s1);                            // Eq. 35 (times dt)
}

// Eqs. A.5, A.4 and A.6-A.7: s at node 1 (tau = 0) and node 5 (tau = 1)
template <int NV, class R>
ADER_DEV void predict_nodal_src(Vec<NV, R>* m, R gm1, R cx, R cy, R cz, PredCtl& ctl, const Src<R>& src,
                                Vec<NV, R>& sdt) {
    const Vec<NV, R> u1 = m[1];
    const Vec<NV, R> u2 = m[1] + 0.5 * m[2], u3 = m[1] + 0.5 * m[3], u4 = m[1] + 0.5 * m[4];
    const Prim<NV, R> p1 = primitives(u1, gm1);
    const Vec<NV, R> s1 = source_at(u1, src);
    const Vec<NV, R> base = u1 - 2.0 * (scale(cx, flux<0>(u2, gm1) - flux_from<0>(u1, p1)) +
                                        scale(cy, flux<1>(u3, gm1) - flux_from<1>(u1, p1)) +
                                        scale(cz, flux<2>(u4, gm1) - flux_from<2>(u1, p1))) +
                            s1 / 3.0;
    iterate_o2(m, ctl, [&](const Vec<NV, R>& m5) {
        const Vec<NV, R> u5 = base + (2.0 / 3.0) * source_at(u1 + m5, src);         // Eq. A.4
        return u5 - u1;                                                              // Eq. A.6
    });
    sdt = 0.5 * (s1 + source_at(u1 + m[5], src));                                   // Eq. A.7 (times dt)
}

// Eqs. 58-59 and D.3-D.5: composing D.4 with D.5, <F> is the mean of the flux
// at the four tau = 1/2 facial nodes (node 5 enters only through the time mode).
template <int D, int NV, class R>
ADER_DEV void face(const Vec<NV, R>* p, R gm1, Vec<NV, R>& ub, Vec<NV, R>& avg, Vec<NV, R>& Fa) {
    ub = p[1] + 0.5 * (p[2] + p[5]);
    avg = ub;
    const Vec<NV, R> q1 = ub;
    Fa = 0.25 * (flux<D>(q1 + 0.5 * p[3], gm1) + flux<D>(q1 - 0.5 * p[3], gm1) + flux<D>(q1 + 0.5 * p[4], gm1) +
                 flux<D>(q1 - 0.5 * p[4], gm1));
}

// MHD face: also the edge averages (Eq. 60 for <u>, Eqs. D.4-D.5 for <F>) of
// the field component each edge's EMF needs.  eu/ef slots: t1+, t1-, t2+, t2-
// (t1 < t2 the transverse axes); component 5 + t1 on the t1 edges, 5 + t2 on
// the t2 edges.
template <int D, class R>
ADER_DEV void face_mhd(const Vec<8, R>* p, R gm1, Vec<8, R>& ub, Vec<8, R>& avg, Vec<8, R>& Fa, R* eu, R* ef) {
    constexpr int T1 = D == 0 ? 1 : 0, T2 = D == 2 ? 1 : 2;
    ub = p[1] + 0.5 * (p[2] + p[5]);
    avg = ub;
    const Vec<8, R> t[6] = {ub, ub + 0.5 * p[3], ub - 0.5 * p[3], ub + 0.5 * p[4], ub - 0.5 * p[4], ub + 0.5 * p[5]};
    Vec<8, R> F[6];
#pragma unroll
    for (int n = 1; n <= 5; ++n) F[n] = flux<D>(t[n], gm1);
    Fa = 0.25 * (F[1] + F[2] + F[3] + F[4]);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const int c = 5 + (s == 0 ? T1 : T2);
        const R m2 = F[1][c] - F[2][c], m3 = F[3][c] - F[4][c];
        const R m4 = R(2) * F[5][c] - R(0.5) * (F[1][c] + F[2][c] + F[3][c] + F[4][c]);
        const R af = F[5][c] - m4 + R(0.5) * m4;
        const R half = R(0.5) * (s == 0 ? m2 : m3);
        ef[2 * s] = af + half;
        ef[2 * s + 1] = af - half;
        const R hu = R(0.5) * p[s == 0 ? 3 : 4][c];
        eu[2 * s] = ub[c] + hu;
        eu[2 * s + 1] = ub[c] - hu;
    }
}

// Full edge-averaged states (all eight components; Eq. 60) for the
// linearized edge fluxes.  Slots as in face_mhd.
template <int D, class R>
ADER_DEV void edge_states(const Vec<8, R>* p, const Vec<8, R>& ub, const Vec<8, R>& avg, Vec<8, R>* e) {
    (void)avg;
    e[0] = ub + 0.5 * p[3];
    e[1] = ub - 0.5 * p[3];
    e[2] = ub + 0.5 * p[4];
    e[3] = ub - 0.5 * p[4];
}

// No paired-face form at this order: the faces are evaluated one at a time.
constexpr bool HAS_FACE_PAIR = false;
template <int D, int NV, class R>
ADER_DEV void face_pair(const Vec<NV, R>*, R, Vec<NV, R>*, Vec<NV, R>*, Vec<NV, R>*) {}

}  // namespace o2
}  // namespace ader
