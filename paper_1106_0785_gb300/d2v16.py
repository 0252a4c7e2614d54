"""The paper's D2V16 velocity set and moment matrix M, as the C ABI takes them.

Sec. II, Fig. 1: v_1..v_4 = (+-1, 0) cyclic, v_5..v_8 = (+-1, +-1),
v_9..v_12 = (+-2, 0) cyclic, v_13..v_16 = (+-2, +-2), in the order fixed by
rows m2 (= v_x) and m3 (= v_y) of M.  The rows of M are the SO(2)
irreducible-representation polynomials (Sec. II) evaluated on these
velocities.  mrtlb_create checks both against the kernels' own tables and
rejects anything else.
"""
import numpy as np


def velocities():
    """(16, 2) float64 array (v_x, v_y), paper order."""
    shells = []
    for c, diag in ((1.0, False), (1.0, True), (2.0, False), (2.0, True)):
        if diag:
            shells += [(c, c), (-c, c), (-c, -c), (c, -c)]
        else:
            shells += [(c, 0.0), (0.0, c), (-c, 0.0), (0.0, -c)]
    return np.array(shells, dtype=np.float64)


def moment_matrix():
    """16 x 16 float64 M, M[k, i] = m_{k+1}(v_{i+1}) (all entries exact)."""
    v = velocities()
    vx, vy = v[:, 0], v[:, 1]
    v2 = vx * vx + vy * vy
    c3x = vx ** 3 - 3.0 * vx * vy ** 2          # v^3 cos 3theta
    c3y = 3.0 * vx ** 2 * vy - vy ** 3          # v^3 sin 3theta
    rows = [
        np.ones(16), vx, vy, v2 / 2.0,
        vx * vx - vy * vy, vx * vy, v2 / 2.0 * vx, v2 / 2.0 * vy,
        c3x, c3y, v2 * v2 / 4.0, vx ** 4 - 6.0 * vx ** 2 * vy ** 2 + vy ** 4,
        v2 * (vx * vx - vy * vy), v2 * vx * vy, v2 * c3x, v2 * c3y,
    ]
    return np.ascontiguousarray(np.stack(rows))
