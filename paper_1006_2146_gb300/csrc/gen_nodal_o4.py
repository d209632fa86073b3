"""Generate nodal_o4_coeffs.cuh: the source-free fourth-order nodal ADER-CG update of App. C.

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
derived numbers with rows printed in Eqs. C.2-C.3.

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
    lines += ["}", "", "}  // namespace o4", "}  // namespace ader", ""]
    return "\n".join(lines)


if __name__ == "__main__":
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "nodal_o4_coeffs.cuh")
    with open(out, "w") as fh:
        fh.write(emit())
    print("wrote", out)
