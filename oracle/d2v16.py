"""D2V16 velocity set and the SO(2) moment matrix M (oracle; test infrastructure).

Sec. II, Fig. 1: sixteen velocities on four shells, speed 1 along the axes,
sqrt(2) on the diagonals, speed 2 along the axes and 2*sqrt(2) on the
diagonals.  "Cyclic permutation" leaves the order inside a shell open; the
printed rows m2 (= v_x) and m3 (= v_y) of M fix it: counter-clockwise,
starting on the +x axis (axis shells) or in the first quadrant (diagonal
shells).

The rows of M (Sec. II) are the SO(2) irreducible-representation
polynomials evaluated on the velocity set.  Here M is built from those
polynomials; a test compares the result with the rows as printed in the
paper (a golden fixture), so a slip in either is caught.

Indices are 0-based in code: q = 0..15 is the paper's i = 1..16 and
k = 0..15 is the paper's moment k = 1..16.
"""
from fractions import Fraction
from functools import lru_cache

import numpy as np

NQ = 16


def velocities():
    """(16, 2) int array of (v_x, v_y) in the paper's order (Sec. II, Fig. 1)."""
    v = []
    for c, diagonal in ((1, False), (1, True), (2, False), (2, True)):
        if diagonal:
            v += [(c, c), (-c, c), (-c, -c), (c, -c)]
        else:
            v += [(c, 0), (0, c), (-c, 0), (0, -c)]
    return np.array(v, dtype=np.int64)


def moment_polynomials(vx, vy):
    """The sixteen row polynomials m_1..m_16 of M at one velocity (exact).

    m1 = 1, m2 = vx, m3 = vy, m4 = v^2/2, m5 = vx^2 - vy^2, m6 = vx vy,
    m7 = (v^2/2) vx, m8 = (v^2/2) vy, m9 = vx^3 - 3 vx vy^2,
    m10 = 3 vx^2 vy - vy^3, m11 = v^4/4, m12 = vx^4 - 6 vx^2 vy^2 + vy^4,
    m13 = v^2 (vx^2 - vy^2), m14 = v^2 vx vy, m15 = v^2 m9, m16 = v^2 m10.
    """
    vx = Fraction(int(vx))
    vy = Fraction(int(vy))
    v2 = vx * vx + vy * vy
    m9 = vx ** 3 - 3 * vx * vy ** 2
    m10 = 3 * vx ** 2 * vy - vy ** 3
    return [
        Fraction(1), vx, vy, v2 / 2,
        vx * vx - vy * vy, vx * vy, v2 / 2 * vx, v2 / 2 * vy,
        m9, m10, v2 * v2 / 4, vx ** 4 - 6 * vx ** 2 * vy ** 2 + vy ** 4,
        v2 * (vx * vx - vy * vy), v2 * vx * vy, v2 * m9, v2 * m10,
    ]


def moment_matrix_exact():
    """M as a 16x16 list of Fractions: M[k][i] = m_k(v_i)."""
    v = velocities()
    cols = [moment_polynomials(vx, vy) for vx, vy in v]
    return [[cols[i][k] for i in range(NQ)] for k in range(NQ)]


def invert_exact(a):
    """Inverse of a square Fraction matrix by Gauss-Jordan elimination.

    Raises ZeroDivisionError-free ValueError when the matrix is singular.
    """
    n = len(a)
    aug = [list(row) + [Fraction(int(i == j)) for j in range(n)]
           for i, row in enumerate(a)]
    for col in range(n):
        piv = next((r for r in range(col, n) if aug[r][col] != 0), None)
        if piv is None:
            raise ValueError("singular matrix")
        aug[col], aug[piv] = aug[piv], aug[col]
        p = aug[col][col]
        aug[col] = [x / p for x in aug[col]]
        for r in range(n):
            if r != col and aug[r][col] != 0:
                fac = aug[r][col]
                aug[r] = [x - fac * y for x, y in zip(aug[r], aug[col])]
    return [row[n:] for row in aug]


@lru_cache(maxsize=None)
def _moment_matrix_f64():
    return np.array([[float(x) for x in row] for row in moment_matrix_exact()])


@lru_cache(maxsize=None)
def _moment_matrix_inverse_f64():
    return np.array([[float(x) for x in row]
                     for row in invert_exact(moment_matrix_exact())])


def moment_matrix():
    """M as float64 (entries are small integers or halves/quarters: exact)."""
    return _moment_matrix_f64().copy()


def moment_matrix_inverse():
    """M^-1 as float64, each entry the rounded exact rational."""
    return _moment_matrix_inverse_f64().copy()
