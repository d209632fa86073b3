"""Node sets of the ADER-CG schemes, as printed in the paper.

Space-time nodes are (xi, eta, zeta, tau); facial nodes are (t1, t2, tau) on a
face xi = +-1/2 (t1 = eta, t2 = zeta for an x-face).  Node n of a set is at
position n-1 (the paper numbers from 1).
"""
import numpy as np

h, q, t3 = 0.5, 0.25, 1.0 / 3.0

# Eq. 31: modal, second order (7 symmetric nodes)
MODAL_O2 = [(h, 0, 0, 0), (-h, 0, 0, 0), (0, h, 0, 0), (0, -h, 0, 0),
            (0, 0, h, 0), (0, 0, -h, 0), (0, 0, 0, 1)]

# Eq. 37: modal, third order (20 symmetric nodes)
MODAL_O3 = [(0, 0, 0, 0), (h, h, 0, 0), (h, -h, 0, 0), (h, 0, h, 0), (h, 0, -h, 0),
            (-h, h, 0, 0), (-h, -h, 0, 0), (-h, 0, h, 0), (-h, 0, -h, 0),
            (0, h, h, 0), (0, -h, h, 0), (0, h, -h, 0), (0, -h, -h, 0),
            (h, 0, 0, h), (-h, 0, 0, h), (0, h, 0, h), (0, -h, 0, h),
            (0, 0, h, h), (0, 0, -h, h), (0, 0, 0, 1)]

# Eq. 46: modal, fourth order (42 symmetric nodes)
MODAL_O4 = [(0, 0, 0, 0), (h, 0, 0, 0), (q, 0, 0, 0), (-q, 0, 0, 0), (-h, 0, 0, 0),
            (0, h, 0, 0), (0, q, 0, 0), (0, -q, 0, 0), (0, -h, 0, 0),
            (0, 0, h, 0), (0, 0, q, 0), (0, 0, -q, 0), (0, 0, -h, 0),
            (h, h, h, 0), (h, -h, h, 0), (h, h, -h, 0), (h, -h, -h, 0),
            (-h, h, h, 0), (-h, -h, h, 0), (-h, h, -h, 0), (-h, -h, -h, 0),
            (0, 0, 0, t3), (h, h, 0, t3), (h, -h, 0, t3), (h, 0, h, t3), (h, 0, -h, t3),
            (-h, h, 0, t3), (-h, -h, 0, t3), (-h, 0, h, t3), (-h, 0, -h, t3),
            (0, h, h, t3), (0, -h, h, t3), (0, h, -h, t3), (0, -h, -h, t3),
            (0, 0, 0, 2 * t3), (h, 0, 0, 2 * t3), (-h, 0, 0, 2 * t3), (0, h, 0, 2 * t3),
            (0, -h, 0, 2 * t3), (0, 0, h, 2 * t3), (0, 0, -h, 2 * t3), (0, 0, 0, 1)]

# Eq. A.1: nodal, second order (5 nodes)
NODAL_O2 = [(0, 0, 0, 0), (h, 0, 0, 0), (0, h, 0, 0), (0, 0, h, 0), (0, 0, 0, 1)]

# Eq. B.1: nodal, third order (15 nodes)
NODAL_O3 = [(0, 0, 0, 0), (h, 0, 0, 0), (-h, 0, 0, 0), (0, h, 0, 0), (0, -h, 0, 0),
            (0, 0, h, 0), (0, 0, -h, 0), (0, h, h, 0), (h, 0, h, 0), (h, h, 0, 0),
            (0, 0, 0, h), (h, 0, 0, h), (0, h, 0, h), (0, 0, h, h), (0, 0, 0, 1)]

# Eq. C.1: nodal, fourth order (35 nodes)
NODAL_O4 = [(0, 0, 0, 0), (h, h, h, 0), (h, 0, 0, 0), (-h, 0, 0, 0), (0, h, 0, 0), (0, -h, 0, 0),
            (0, 0, h, 0), (0, 0, -h, 0), (0, h, h, 0), (-h, 0, h, 0), (h, 0, h, 0), (h, -h, 0, 0),
            (h, h, 0, 0), (0, h, -h, 0), (-q, -h, -h, 0), (q, -h, -h, 0),
            (-h, -q, -h, 0), (-h, q, -h, 0), (-h, -h, -q, 0), (-h, -h, q, 0),
            (0, 0, 0, t3), (h, 0, 0, t3), (-h, 0, 0, t3), (0, h, 0, t3), (0, -h, 0, t3),
            (0, 0, h, t3), (0, 0, -h, t3), (0, h, h, t3), (h, 0, h, t3), (h, h, 0, t3),
            (0, 0, 0, 2 * t3), (h, 0, 0, 2 * t3), (0, h, 0, 2 * t3), (0, 0, h, 2 * t3), (0, 0, 0, 1)]

# Eq. D.1, D.6, D.11: one-sided facial nodes (t1, t2, tau) on the face xi = +1/2
# (the same (t1, t2, tau) are used on the face xi = -1/2, App. D).
FACE_O2 = [(h, 0, h), (-h, 0, h), (0, h, h), (0, -h, h), (0, 0, 1)]
FACE_O3 = [(0, 0, 0), (h, h, 0), (-h, h, 0), (h, -h, 0), (-h, -h, 0),
           (h, 0, h), (-h, 0, h), (0, h, h), (0, -h, h), (0, 0, 1)]
FACE_O4 = [(0, 0, 0), (h, 0, 0), (q, 0, 0), (-q, 0, 0), (-h, 0, 0),
           (0, h, 0), (0, q, 0), (0, -q, 0), (0, -h, 0),
           (h, h, 0), (-h, h, 0), (h, -h, 0), (-h, -h, 0),
           (0, 0, t3), (h, h, t3), (-h, h, t3), (h, -h, t3), (-h, -h, t3),
           (0, 0, 2 * t3), (h, 0, 2 * t3), (-h, 0, 2 * t3), (0, h, 2 * t3), (0, -h, 2 * t3),
           (0, 0, 1)]

MODAL = {2: MODAL_O2, 3: MODAL_O3, 4: MODAL_O4}
NODAL = {2: NODAL_O2, 3: NODAL_O3, 4: NODAL_O4}
FACE = {2: FACE_O2, 3: FACE_O3, 4: FACE_O4}


def as_array(nodes):
    return np.asarray(nodes, dtype=np.float64)
