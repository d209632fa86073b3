"""Generate nodal_o4_coeffs.cuh: the fourth-order nodal ADER-CG update of App. C.

The nodal scheme evolves the values at the 35 nodes of Eq. C.1.  Without
source terms its update is linear in the scaled nodal fluxes: the flux
polynomial is the interpolant through the nodes (one node per mode of
Eq. 16), and du/dtau = -(f_xi + g_eta + h_zeta) fixes the evolutionary modes.
For each evolutionary node k = 21..35,
    u_k = u_base(k) + sum_{j<=20} (c^f_kj f_j + c^g_kj g_j + c^h_kj h_j)     (q-term, Eq. C.2)
                    + sum_{j>=21} (c^f_kj f_j + c^g_kj g_j + c^h_kj h_j)     (Eq. C.3)
where base(k) is the tau = 0 node at the same spatial point.  The paper
prints these coefficients as integers over 53865 .. 646380; this script
derives them exactly (rational arithmetic) and writes them as sparse CUDA
statements.  `coefficients()` is also used by a CPU test that compares the
derived numbers with rows printed in Eqs. C.2-C.3.  `source_coefficients()`
adds the non-stiff source terms of Eqs. C.2-C.3 (a Galerkin projection of the
source interpolant, see there) and the weights of S-bar (Eq. C.6).

Run:  python gen_nodal_o4.py   (rewrites nodal_o4_coeffs.cuh next to this file)
"""
import os
from fractions import Fraction as Fr

H, Q, T3 = Fr(1, 2), Fr(1, 4), Fr(1, 3)

# Eq. C.1
NODES = [(0, 0, 0, 0), (H, H, H, 0), (H, 0, 0, 0), (-H, 0, 0, 0), (0, H, 0, 0), (0, -H, 0, 0),
         (0, 0, H, 0), (0, 0, -H, 0), (0, H, H, 0), (-H, 0, H, 0), (H, 0, H, 0), (H, -H, 0, 0),
         (H, H, 0, 0), (0, H, -H, 0), (-Q, -H, -H, 0), (Q, -H, -H, 0),
         (-H, -Q, -H, 0), (-H, Q, -H, 0), (-H, -H, -Q, 0), (-H, -H, Q, 0),
         (0, 0, 0, T3), (H, 0, 0, T3), (-H, 0, 0, T3), (0, H, 0, T3), (0, -H, 0, T3),
         (0, 0, H, T3), (0, 0, -H, T3), (0, H, H, T3), (H, 0, H, T3), (H, H, 0, T3),
         (0, 0, 0, 2 * T3), (H, 0, 0, 2 * T3), (0, H, 0, 2 * T3), (0, 0, H, 2 * T3), (0, 0, 0, 1)]

# Eq. 16: exponents (a, b, c, d) of P_a(xi) P_b(eta) P_c(zeta) tau^d
MODES = [(0, 0, 0, 0), (1, 0, 0, 0), (0, 1, 0, 0), (0, 0, 1, 0), (2, 0, 0, 0), (0, 2, 0, 0), (0, 0, 2, 0),
         (1, 1, 0, 0), (0, 1, 1, 0), (1, 0, 1, 0), (3, 0, 0, 0), (0, 3, 0, 0), (0, 0, 3, 0),
         (2, 1, 0, 0), (2, 0, 1, 0), (1, 2, 0, 0), (0, 2, 1, 0), (1, 0, 2, 0), (0, 1, 2, 0), (1, 1, 1, 0),
         (0, 0, 0, 1), (0, 0, 0, 2), (0, 0, 0, 3), (1, 0, 0, 1), (0, 1, 0, 1), (0, 0, 1, 1),
         (1, 0, 0, 2), (0, 1, 0, 2), (0, 0, 1, 2), (2, 0, 0, 1), (0, 2, 0, 1), (0, 0, 2, 1),
         (1, 1, 0, 1), (0, 1, 1, 1), (1, 0, 1, 1)]

# Eq. 9, ascending powers
PPOLY = [[Fr(1)], [Fr(0), Fr(1)], [Fr(-1, 12), Fr(0), Fr(1)], [Fr(0), Fr(-3, 20), Fr(0), Fr(1)]]


def _p(a, x):
    return sum(c * x ** i for i, c in enumerate(PPOLY[a]))


def _phi(mode, pt):
    a, b, c, d = mode
    return _p(a, pt[0]) * _p(b, pt[1]) * _p(c, pt[2]) * pt[3] ** d


def _dP(a):
    """d/dx P_a as a combination {a': coef} of P's (P_n monic of degree n)."""
    poly = [i * c for i, c in enumerate(PPOLY[a])][1:]
    out = {}
    for deg in range(len(poly) - 1, -1, -1):
        c = poly[deg]
        if c != 0:
            out[deg] = c
            for i, pc in enumerate(PPOLY[deg]):
                poly[i] -= c * pc
    return out


def _inverse(M):
    n = len(M)
    A = [row[:] + [Fr(int(i == j)) for j in range(n)] for i, row in enumerate(M)]
    for col in range(n):
        piv = next(r for r in range(col, n) if A[r][col] != 0)
        A[col], A[piv] = A[piv], A[col]
        pv = A[col][col]
        A[col] = [x / pv for x in A[col]]
        for r in range(n):
            if r != col and A[r][col] != 0:
                f = A[r][col]
                A[r] = [x - f * y for x, y in zip(A[r], A[col])]
    return [row[n:] for row in A]


def coefficients():
    """C[d][k][j] (exact): response of node k (1-based, 21..35) to scaled flux d at node j (1-based)."""
    n = len(NODES)
    V = [[_phi(m, p) for m in MODES] for p in NODES]
    Vi = _inverse(V)
    idx = {m: i for i, m in enumerate(MODES)}
    C = [[[Fr(0)] * (n + 1) for _ in range(n + 1)] for _ in range(3)]
    for d in range(3):
        for j in range(n):
            fm = [Vi[k][j] for k in range(n)]              # flux modes of a unit value at node j
            r = [Fr(0)] * n                                 # -d(flux)/d(coordinate d) in the basis
            for k, m in enumerate(MODES):
                if m[d] == 0 or fm[k] == 0:
                    continue
                for a2, c in _dP(m[d]).items():
                    m2 = list(m)
                    m2[d] = a2
                    r[idx[tuple(m2)]] -= c * fm[k]
            evo = [Fr(0)] * n                               # evolutionary modes: tau-derivative matching
            for k, (a, b, c, dd) in enumerate(MODES):
                if dd >= 1:
                    evo[k] = r[idx[(a, b, c, dd - 1)]] / dd
            for node in range(20, n):
                C[d][node + 1][j + 1] = sum(V[node][k] * evo[k] for k in range(n) if evo[k] != 0)
    return C


def _int1d(a, b):
    """Exact integral over [-1/2, 1/2] of P_a P_b."""
    prod = [Fr(0)] * (len(PPOLY[a]) + len(PPOLY[b]) - 1)
    for i, ca in enumerate(PPOLY[a]):
        for j, cb in enumerate(PPOLY[b]):
            prod[i + j] += ca * cb
    return sum(c * (Fr(1, 2) ** (p + 1) - Fr(-1, 2) ** (p + 1)) / (p + 1) for p, c in enumerate(prod))


def source_coefficients():
    """(CS, W) exact.  CS[k][j]: response of node k (21..35) to the scaled source s = dt S at node j
    (1..35); W[j]: weight of node j in the space-time average of the source polynomial (dt S-bar).

    With a source, du/dtau = -div f + s holds in the Galerkin sense with the Lagrange polynomials of the
    nodes with tau > 0 as test functions (the source polynomial is the interpolant through the nodes);
    the flux part stays the derivative matching of coefficients(), its exact solution."""
    n = len(NODES)
    V = [[_phi(m, p) for m in MODES] for p in NODES]
    Vi = _inverse(V)
    idx = {m: i for i, m in enumerate(MODES)}
    E = [k for k, m in enumerate(MODES) if m[3] >= 1]
    M = [[Fr(0)] * n for _ in range(n)]
    for i, mi in enumerate(MODES):
        for j, mj in enumerate(MODES):
            sp = _int1d(mi[0], mj[0]) * _int1d(mi[1], mj[1]) * _int1d(mi[2], mj[2])
            if sp != 0:
                M[i][j] = sp * Fr(1, mi[3] + mj[3] + 1)
    T = [[Fr(0)] * n for _ in range(n)]                     # T[j][k]: mode j in d(phi_k)/d(tau)
    for k, (a, b, c, d) in enumerate(MODES):
        if d >= 1:
            T[idx[(a, b, c, d - 1)]][k] = Fr(d)
    evo_nodes = [q for q in range(n) if NODES[q][3] > 0]
    Psi = [[Vi[i][q] for q in evo_nodes] for i in range(n)]  # Lagrange polynomials of the tau > 0 nodes
    PM = [[sum(Psi[i][r] * M[i][j] for i in range(n) if Psi[i][r] != 0) for j in range(n)]
          for r in range(len(evo_nodes))]
    A = [[sum(PM[r][j] * T[j][E[c]] for j in range(n) if T[j][E[c]] != 0) for c in range(len(E))]
         for r in range(len(evo_nodes))]
    Ai = _inverse(A)
    # evolutionary modes of a unit source value at node q: Ai PM Vi[:, q]
    CS = [[Fr(0)] * (n + 1) for _ in range(n + 1)]
    for q in range(n):
        sm = [Vi[k][q] for k in range(n)]
        b = [sum(PM[r][j] * sm[j] for j in range(n) if sm[j] != 0) for r in range(len(evo_nodes))]
        evo = [sum(Ai[c][r] * b[r] for r in range(len(evo_nodes))) for c in range(len(E))]
        for node in range(20, n):
            CS[node + 1][q + 1] = sum(V[node][E[c]] * evo[c] for c in range(len(E)))
    avg = []
    for (a, b, c, d) in MODES:
        avg.append(_int1d(a, 0) * _int1d(b, 0) * _int1d(c, 0) * Fr(1, d + 1))
    W = [Fr(0)] + [sum(avg[k] * Vi[k][q] for k in range(n)) for q in range(n)]
    return CS, W


def base_node(k):
    """The tau = 0 node at the spatial point of node k."""
    x = NODES[k - 1][:3]
    return next(i + 1 for i, p in enumerate(NODES[:20]) if p[:3] == x)


def _terms(C, k, lo, hi, f_name, idx_shift):
    out = []
    for d, arr in enumerate(("f", "g", "h")):
        for j in range(lo, hi + 1):
            c = C[d][k][j]
            if c != 0:
                out.append("%.17g * %s[%d]" % (float(c), arr, j - idx_shift))
    return out


def emit():
    C = coefficients()
    lines = [
        "// Generated by gen_nodal_o4.py: source-free fourth-order nodal update (App. C, Eqs. C.2-C.3).",
        "// u_k = u_base(k) + sum over tau = 0 nodes (q-term) + sum over tau > 0 nodes, k = 21..35.",
        "// Coefficients derived exactly from Lagrange interpolation on the nodes of Eq. C.1 and",
        "// du/dtau = -div f in the basis of Eq. 16; do not edit by hand.",
        "#pragma once",
        '#include "common.cuh"',
        "namespace ader {",
        "namespace o4 {",
        "",
        "// qt[k-21] = u[base(k)] + tau = 0 flux terms; f, g, h indexed by node 1..20",
        "template <int NV, class R>",
        "ADER_DEV void nodal_o4_qterms(const Vec<NV, R>* u, const Vec<NV, R>* f, const Vec<NV, R>* g,",
        "                              const Vec<NV, R>* h, Vec<NV, R>* qt) {",
    ]
    for k in range(21, 36):
        t = _terms(C, k, 1, 20, None, 0)
        lines.append("    qt[%d] = u[%d]%s;" % (k - 21, base_node(k), "".join("\n        + " + s for s in t)))
    lines += ["}", "",
              "// e[k-21] = value at node k before the first iteration: the tau = 0 value at its spatial",
              "// point plus the evolutionary modes m[21..35] (the initial guess) evaluated there",
              "template <int NV, class R>",
              "ADER_DEV void nodal_o4_initial(const Vec<NV, R>* u, const Vec<NV, R>* m, Vec<NV, R>* e) {"]
    for k in range(21, 36):
        terms = []
        for j, mode in enumerate(MODES):
            if mode[3] == 0:
                continue
            c = _phi(mode, NODES[k - 1])
            if c != 0:
                terms.append("%.17g * m[%d]" % (float(c), j + 1))
        lines.append("    e[%d] = u[%d]%s;" % (k - 21, base_node(k), "".join(" + " + t for t in terms)))
    lines += ["}", "",
              "// one Picard step: e[k-21] = qt[k-21] + tau > 0 flux terms; f, g, h indexed by node - 21",
              "template <int NV, class R>",
              "ADER_DEV void nodal_o4_update(const Vec<NV, R>* qt, const Vec<NV, R>* f, const Vec<NV, R>* g,",
              "                              const Vec<NV, R>* h, Vec<NV, R>* e) {"]
    for k in range(21, 36):
        t = _terms(C, k, 21, 35, None, 21)
        assert all("[14]" not in s for s in t), "node 35 flux must not enter the update"
        lines.append("    e[%d] = qt[%d]%s;" % (k - 21, k - 21, "".join("\n        + " + s for s in t)))
    CS, W = source_coefficients()
    lines += ["}", "",
              "// the source terms of Eq. C.2: qt[k-21] += tau = 0 node sources s[1..20] (s = dt S)",
              "template <int NV, class R>",
              "ADER_DEV void nodal_o4_qterms_src(const Vec<NV, R>* s, Vec<NV, R>* qt) {"]
    for k in range(21, 36):
        t = ["%.17g * s[%d]" % (float(CS[k][j]), j) for j in range(1, 21) if CS[k][j] != 0]
        if t:
            lines.append("    qt[%d] += %s;" % (k - 21, "\n        + ".join(t)))
    lines += ["}", "",
              "// the source terms of Eq. C.3: e[k-21] += tau > 0 node sources s[node - 21] of the current iterate",
              "template <int NV, class R>",
              "ADER_DEV void nodal_o4_update_src(const Vec<NV, R>* s, Vec<NV, R>* e) {"]
    for k in range(21, 36):
        t = ["%.17g * s[%d]" % (float(CS[k][j]), j - 21) for j in range(21, 36) if CS[k][j] != 0]
        if t:
            lines.append("    e[%d] += %s;" % (k - 21, "\n        + ".join(t)))
    lines += ["}", "",
              "// dt S-bar (Eq. C.6): the space-time average of the source interpolant; s0 indexed by node",
              "// 1..20, s1 by node - 21",
              "template <int NV, class R>",
              "ADER_DEV Vec<NV, R> nodal_o4_sbar(const Vec<NV, R>* s0, const Vec<NV, R>* s1) {"]
    t = ["%.17g * s0[%d]" % (float(W[j]), j) for j in range(1, 21) if W[j] != 0]
    t += ["%.17g * s1[%d]" % (float(W[j]), j - 21) for j in range(21, 36) if W[j] != 0]
    lines.append("    return %s;" % "\n        + ".join(t))
    lines += ["}", "", "}  // namespace o4", "}  // namespace ader", ""]
    return "\n".join(lines)


if __name__ == "__main__":
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "nodal_o4_coeffs.cuh")
    with open(out, "w") as fh:
        fh.write(emit())
    print("wrote", out)
