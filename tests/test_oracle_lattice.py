"""Pins of the oracle's velocity set and moment matrix (Sec. II, Fig. 1)."""
import os
from fractions import Fraction

import numpy as np

from oracle import d2v16

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _paper_rows():
    rows = []
    with open(os.path.join(GOLDEN, "paper_M_rows.txt")) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([Fraction(tok) for tok in line.split()])
    return rows


def test_velocity_set_shells_and_pairs():
    v = d2v16.velocities()
    speeds2 = (v ** 2).sum(1)
    # four shells of four: |v|^2 = 1, 2, 4, 8 (Fig. 1)
    assert list(speeds2) == [1] * 4 + [2] * 4 + [4] * 4 + [8] * 4
    # every velocity has its opposite in the set, within its shell
    for q in range(16):
        opp = [p for p in range(16) if (v[p] == -v[q]).all()]
        assert len(opp) == 1 and opp[0] // 4 == q // 4
    # the lattice is symmetric: odd moments vanish, even ones isotropic
    assert (v.sum(0) == 0).all()


def test_moment_matrix_equals_printed_rows():
    printed = _paper_rows()
    assert len(printed) == 16 and all(len(r) == 16 for r in printed)
    assert d2v16.moment_matrix_exact() == printed


def test_rows_two_three_fix_velocity_order():
    printed = np.array([[float(x) for x in r] for r in _paper_rows()])
    v = d2v16.velocities()
    assert (printed[1] == v[:, 0]).all()
    assert (printed[2] == v[:, 1]).all()


def test_exact_inverse():
    M = d2v16.moment_matrix_exact()
    Mi = d2v16.invert_exact(M)
    n = 16
    for i in range(n):
        for j in range(n):
            s = sum(M[i][k] * Mi[k][j] for k in range(n))
            assert s == (1 if i == j else 0)
    Mf = d2v16.moment_matrix()
    Mif = d2v16.moment_matrix_inverse()
    assert np.abs(Mf @ Mif - np.eye(16)).max() < 1e-14
    assert np.abs(Mif @ Mf - np.eye(16)).max() < 1e-14
    # the float inverse agrees with an independent LU solve
    assert np.allclose(Mif, np.linalg.inv(Mf), rtol=0, atol=1e-12)
