"""Flux-mode extraction rules of the modal predictor and of the facial quadrature.

These are rules, not definitions: the node sets of the modal scheme (Eqs. 31,
37, 46) and of the facial quadrature at second and fourth order (Eqs. D.1,
D.11) hold more nodes than there are modes, so the paper fixes one linear
combination per mode.  The oracle applies them literally.  Each function takes
nodal values with the node index on the first axis (``fb[n-1]`` is the value
at node n) and returns a dict {mode number (1-based): array}.

Pinned in tests/test_oracle_extraction.py: every rule returns the exact modes
of any flux polynomial that lies in the span of the basis.
"""


# ----------------------------------------------------------------------------- modal, Sec. IV
def modal_o2(f, g, h):
    """Eq. 33."""
    return ({2: f[0] - f[1]},
            {3: g[2] - g[3]},
            {4: h[4] - h[5]})


def modal_o3(f, g, h):
    """Eqs. 40 (x), 41 (y), 42 (z)."""
    F = lambda n: f[n - 1]
    G = lambda n: g[n - 1]
    H = lambda n: h[n - 1]
    fx = {}
    q1 = F(2) + F(3) + F(4) + F(5)
    q2 = F(6) + F(7) + F(8) + F(9)
    q3 = F(10) + F(11) + F(12) + F(13)
    fx[2] = 0.25 * (q1 - q2)
    fx[5] = 0.5 * (q1 + q2 - q3) - 2.0 * F(1)
    fx[8] = F(2) - F(3) - F(6) + F(7)
    fx[10] = F(4) - F(5) - F(8) + F(9)
    fx[13] = 2.0 * (F(14) - F(15) - fx[2])
    gy = {}
    q4 = G(2) + G(6) + G(10) + G(12)
    q5 = G(3) + G(7) + G(11) + G(13)
    q6 = G(4) + G(5) + G(8) + G(9)
    gy[3] = 0.25 * (q4 - q5)
    gy[6] = 0.5 * (q4 + q5 - q6) - 2.0 * G(1)
    gy[8] = G(2) - G(3) - G(6) + G(7)
    gy[9] = G(10) - G(11) - G(12) + G(13)
    gy[14] = 2.0 * (G(16) - G(17) - gy[3])
    hz = {}
    q7 = H(4) + H(8) + H(10) + H(11)
    q8 = H(5) + H(9) + H(12) + H(13)
    q9 = H(2) + H(3) + H(6) + H(7)
    hz[4] = 0.25 * (q7 - q8)
    hz[7] = 0.5 * (q7 + q8 - q9) - 2.0 * H(1)
    hz[9] = H(10) - H(11) - H(12) + H(13)
    hz[10] = H(4) - H(5) - H(8) + H(9)
    hz[15] = 2.0 * (H(18) - H(19) - hz[4])
    return fx, gy, hz


def _o4_common_q(X):
    """The temporaries q1..q9 shared by Eqs. 49, 50 and 51 (same nodes for every flux)."""
    q = {}
    q[1] = X(14) + X(15) + X(16) + X(17)
    q[2] = X(18) + X(19) + X(20) + X(21)
    q[3] = X(14) + X(16) + X(18) + X(20)
    q[4] = X(15) + X(17) + X(19) + X(21)
    q[5] = X(14) + X(15) + X(18) + X(19)
    q[6] = X(16) + X(17) + X(20) + X(21)
    q[7] = X(23) + X(24) - X(25) - X(26) - X(27) - X(28) + X(29) + X(30)
    q[8] = X(23) + X(27) - X(24) - X(28) - X(31) - X(33) + X(32) + X(34)
    q[9] = X(25) + X(29) - X(26) - X(30) - X(31) - X(32) + X(33) + X(34)
    return q


def _o4_mixed(X, q, m):
    """Modes 14-20 of Eqs. 49-51; the paper prints the same rule for f, g and h."""
    m[14] = q[8] + 0.5 * (q[3] - q[4]) - 2.0 * (X(6) - X(9))
    m[15] = q[9] + 0.5 * (q[5] - q[6]) - 2.0 * (X(10) - X(13))
    m[16] = q[7] + 0.5 * (q[1] - q[2]) - 2.0 * (X(2) - X(5))
    m[17] = -2.0 * q[9] + m[15]
    m[18] = -2.0 * q[7] + m[16]
    m[19] = -2.0 * q[8] + m[14]
    m[20] = X(14) - X(15) - X(16) + X(17) - X(18) + X(19) + X(20) - X(21)


def modal_o4(f, g, h):
    """Eqs. 49 (x), 50 (y), 51 (z)."""
    F = lambda n: f[n - 1]
    G = lambda n: g[n - 1]
    H = lambda n: h[n - 1]
    # x-flux, Eq. 49
    q = _o4_common_q(F)
    q10 = F(23) + F(24) + F(25) + F(26) - F(27) - F(28) - F(29) - F(30)
    fx = {}
    fx[5] = 2.0 * (F(2) - 2.0 * F(1) + F(5))
    fx[8] = 0.5 * (F(14) - F(15) + F(16) - F(17) - F(18) + F(19) - F(20) + F(21))
    fx[10] = 0.5 * (F(14) + F(15) - F(16) - F(17) - F(18) - F(19) + F(20) + F(21))
    fx[11] = 16.0 * (F(2) - 2.0 * F(3) + 2.0 * F(4) - F(5)) / 3.0
    fx[2] = 2.0 * (F(2) - F(5)) / 3.0 - 0.1 * fx[11] + (q[1] - q[2]) / 12.0
    _o4_mixed(F, q, fx)
    fx[27] = 1.125 * (q[1] - q[2]) + 4.5 * (F(36) - F(37)) - 2.25 * q10
    fx[24] = 3.0 * (F(36) - F(37)) - 0.75 * q10 + 0.375 * (fx[16] + fx[18]) - fx[27]
    fx[30] = 3.0 * (F(36) - 2.0 * F(35) + F(37)) - 1.5 * fx[5]
    fx[33] = 3.0 * (F(23) - F(27) - F(24) + F(28)) - 3.0 * fx[8]
    fx[35] = 3.0 * (F(25) - F(29) - F(26) + F(30)) - 3.0 * fx[10]
    # y-flux, Eq. 50
    q = _o4_common_q(G)
    q11 = G(23) - G(24) + G(27) - G(28) + G(31) - G(32) + G(33) - G(34)
    gy = {}
    gy[6] = 2.0 * (G(6) - 2.0 * G(1) + G(9))
    gy[8] = 0.5 * (G(14) - G(15) + G(16) - G(17) - G(18) + G(19) - G(20) + G(21))
    gy[9] = 0.5 * (G(14) - G(15) - G(16) + G(17) + G(18) - G(19) - G(20) + G(21))
    gy[12] = 16.0 * (G(6) - 2.0 * G(7) + 2.0 * G(8) - G(9)) / 3.0
    gy[3] = 2.0 * (G(6) - G(9)) / 3.0 - 0.1 * gy[12] + (q[3] - q[4]) / 12.0
    _o4_mixed(G, q, gy)
    gy[28] = 1.125 * (q[3] - q[4]) + 4.5 * (G(38) - G(39)) - 2.25 * q11
    gy[25] = 3.0 * (G(38) - G(39)) - 0.75 * q11 + 0.375 * (gy[14] + gy[19]) - gy[28]
    gy[31] = 3.0 * (G(38) - 2.0 * G(35) + G(39)) - 1.5 * gy[6]
    gy[33] = 3.0 * (G(23) - G(27) - G(24) + G(28)) - 3.0 * gy[8]
    gy[34] = 3.0 * (G(31) - G(32) - G(33) + G(34)) - 3.0 * gy[9]
    # z-flux, Eq. 51
    q = _o4_common_q(H)
    q12 = H(25) - H(26) + H(29) - H(30) + H(31) + H(32) - H(33) - H(34)
    hz = {}
    hz[7] = 2.0 * (H(10) - 2.0 * H(1) + H(13))
    hz[9] = 0.5 * (H(14) - H(15) - H(16) + H(17) + H(18) - H(19) - H(20) + H(21))
    hz[10] = 0.5 * (H(14) + H(15) - H(16) - H(17) - H(18) - H(19) + H(20) + H(21))
    hz[13] = 16.0 * (H(10) - 2.0 * H(11) + 2.0 * H(12) - H(13)) / 3.0
    hz[4] = 2.0 * (H(10) - H(13)) / 3.0 - 0.1 * hz[13] + (q[5] - q[6]) / 12.0
    _o4_mixed(H, q, hz)
    hz[29] = 1.125 * (q[5] - q[6]) + 4.5 * (H(40) - H(41)) - 2.25 * q12
    hz[26] = 3.0 * (H(40) - H(41)) - 0.75 * q12 + 0.375 * (hz[15] + hz[17]) - hz[29]
    hz[32] = 3.0 * (H(40) - 2.0 * H(35) + H(41)) - 1.5 * hz[7]
    hz[34] = 3.0 * (H(31) - H(32) - H(33) + H(34)) - 3.0 * hz[9]
    hz[35] = 3.0 * (H(25) - H(26) - H(29) + H(30)) - 3.0 * hz[10]
    return fx, gy, hz


MODAL = {2: modal_o2, 3: modal_o3, 4: modal_o4}

# Flux modes each modal rule must deliver: every mode whose basis function
# depends on the flux's own direction (those are the ones d/dxi does not kill).
NEEDED = {
    2: ({2}, {3}, {4}),
    3: ({2, 5, 8, 10, 13}, {3, 6, 8, 9, 14}, {4, 7, 9, 10, 15}),
    4: ({2, 5, 8, 10, 11, 14, 15, 16, 18, 20, 24, 27, 30, 33, 35},
        {3, 6, 8, 9, 12, 14, 16, 17, 19, 20, 25, 28, 31, 33, 34},
        {4, 7, 9, 10, 13, 15, 17, 18, 19, 20, 26, 29, 32, 34, 35}),
}


# ----------------------------------------------------------------------------- facial, App. D
def face_o2(f):
    """Eq. D.4: modes of the facial flux polynomial Eq. D.2 from the 5 nodes of Eq. D.1."""
    m = {}
    m[2] = f[0] - f[1]
    m[3] = f[2] - f[3]
    m[4] = 2.0 * f[4] - 0.5 * (f[0] + f[1] + f[2] + f[3])
    m[1] = f[4] - m[4]
    return m


def face_o4(f):
    """Eq. D.14: modes of Eq. D.12 from the 24 nodes of Eq. D.11."""
    F = lambda n: f[n - 1]
    m = {}
    q1 = 3.0 * (F(20) - F(21)) - 1.5 * (F(15) - F(16) + F(17) - F(18))
    q2 = 1.5 * (F(20) - F(21) - F(2) + F(5))
    q3 = 3.0 * (F(22) - F(23)) - 1.5 * (F(15) + F(16) - F(17) - F(18))
    q4 = 1.5 * (F(22) - F(23) - F(6) + F(9))
    m[1] = (2.0 * F(1) + F(2) + F(5) + F(6) + F(9)) / 6.0
    m[4] = 2.0 * (F(2) - 2.0 * F(1) + F(5))
    m[5] = 2.0 * (F(6) - 2.0 * F(1) + F(9))
    m[6] = F(10) - F(11) - F(12) + F(13)
    m[7] = 16.0 * (F(2) - 2.0 * F(3) + 2.0 * F(4) - F(5)) / 3.0
    m[8] = 16.0 * (F(6) - 2.0 * F(7) + 2.0 * F(8) - F(9)) / 3.0
    m[9] = 2.0 * (F(10) - 2.0 * F(6) + F(11) - F(12) + 2.0 * F(9) - F(13))
    m[10] = 2.0 * (F(10) - 2.0 * F(2) + F(12) - F(11) + 2.0 * F(5) - F(13))
    m[2] = F(2) - F(5) + m[10] / 12.0 - 0.1 * m[7]
    m[3] = F(6) - F(9) + m[9] / 12.0 - 0.1 * m[8]
    m[13] = 4.5 * (F(24) - F(1)) - 13.5 * (F(19) - F(14))
    m[12] = 2.25 * (F(24) - F(19) - F(14) + F(1) - 2.0 * m[13] / 3.0)
    m[11] = (1.5 * F(24) - 2.5 * F(14) + 0.25 * (F(15) + F(16) + F(17) + F(18))
             - 0.25 * m[4] - 0.25 * m[5] - 4.0 * m[12] / 3.0 - 13.0 * m[13] / 9.0)
    m[14] = 3.0 * q2 - 2.0 * q1 - 1.5 * m[10]
    m[16] = 3.0 * (q1 - q2) + 2.25 * m[10]
    m[15] = 3.0 * q4 - 2.0 * q3 - 1.5 * m[9]
    m[17] = 3.0 * (q3 - q4) + 2.25 * m[9]
    m[18] = 3.0 * (F(20) - 2.0 * F(19) + F(21)) - 1.5 * m[4]
    m[19] = 3.0 * (F(22) - 2.0 * F(19) + F(23)) - 1.5 * m[5]
    m[20] = 3.0 * (F(15) - F(16) - F(17) + F(18)) - 3.0 * m[6]
    return m
