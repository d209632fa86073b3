// Second order: ADER-CG predictor (modal Sec. IV.1, nodal App. A) and the x+
// face quantities (Sec. V.1, App. D).  Modes m[1..5] (Eq. 14).
#pragma once
#include "common.cuh"
#include "modes.cuh"

namespace ader {
namespace o2 {

template <class R> using V = Vec<5, R>;

// Eqs. 31-33 and 30 (one iteration, no sources)
template <class R>
ADER_DEV void predict_modal(V<R>* m, R gm1, R cx, R cy, R cz, int n_iter) {
    const V<R> u1 = m[1] + 0.5 * m[2], u2 = m[1] - 0.5 * m[2];
    const V<R> u3 = m[1] + 0.5 * m[3], u4 = m[1] - 0.5 * m[3];
    const V<R> u5 = m[1] + 0.5 * m[4], u6 = m[1] - 0.5 * m[4];
    const V<R> F2 = scale(cx, flux<0>(u1, gm1) - flux<0>(u2, gm1));
    const V<R> G3 = scale(cy, flux<1>(u3, gm1) - flux<1>(u4, gm1));
    const V<R> H4 = scale(cz, flux<2>(u5, gm1) - flux<2>(u6, gm1));
    m[5] = n_iter > 0 ? -(F2 + G3 + H4) : m[5];
}

// Eqs. A.5, A.4 (h term at node 4, the zeta node of Eq. A.1) and A.6
template <class R>
ADER_DEV void predict_nodal(V<R>* m, R gm1, R cx, R cy, R cz, int n_iter) {
    const V<R> u1 = m[1];
    const V<R> u2 = m[1] + 0.5 * m[2], u3 = m[1] + 0.5 * m[3], u4 = m[1] + 0.5 * m[4];
    const Prim<R> p1 = primitives(u1, gm1);
    const V<R> u5 = u1 - 2.0 * (scale(cx, flux<0>(u2, gm1) - flux_from<0>(u1, p1)) +
                                scale(cy, flux<1>(u3, gm1) - flux_from<1>(u1, p1)) +
                                scale(cz, flux<2>(u4, gm1) - flux_from<2>(u1, p1)));
    m[5] = n_iter > 0 ? u5 - u1 : m[5];
}

// Eqs. 58-59 and D.3-D.5: composing D.4 with D.5, <F> is the mean of the flux
// at the four tau = 1/2 facial nodes (node 5 enters only through the time mode).
template <int D, class R>
ADER_DEV void face(const V<R>* p, R gm1, V<R>& ub, V<R>& avg, V<R>& Fa) {
    ub = p[1] + 0.5 * (p[2] + p[5]);
    avg = ub;
    const V<R> q1 = ub;
    Fa = 0.25 * (flux<D>(q1 + 0.5 * p[3], gm1) + flux<D>(q1 - 0.5 * p[3], gm1) + flux<D>(q1 + 0.5 * p[4], gm1) +
                 flux<D>(q1 - 0.5 * p[4], gm1));
}

}  // namespace o2
}  // namespace ader
