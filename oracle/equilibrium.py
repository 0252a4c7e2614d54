"""Macroscopic recovery and equilibrium moments (oracle; test infrastructure).

Sec. II: the conserved moments are f^_1 = rho, f^_2 = j_x, f^_3 = j_y,
f^_4 = e = rho (T + u^2/2) with R = 1 (Sec. IV works in units where R = 1).
Eqs. 14a-14i give the equilibria of the non-conserved moments
k = 5..11, 13, 14.  The three "versions" for k = 12, 15, 16 (Sec. II, after
Eq. 5):
  version 1: all three zero;
  version 2: f^12 = 0, f^15 = rho ux (-4 + 10 T + 5 ux^2 - 5 uy^2),
             f^16 = rho uy (4 - 10 T + 5 ux^2 - 5 uy^2);
  version 3: f^k = sum_i M_ki f_i^max with
             f_i^max = rho / (2 pi T) exp(-(v_i - u)^2 / (2 T)).

All functions broadcast over arrays of any shape and accept complex input
(complex-step differentiation).

Parity unpinned: the values of the version-2 formulas.  The paper derives
them from the requirement that the model reduce to an earlier
single-relaxation-time model (Chen 1994), which is not part of the paper,
so their values are pinned only as the text states them.  What the paper
does fix about them is checked: they leave the conserved moments untouched
and the collision conserving; they turn into each other under the lattice's
90-degree rotation and reflections (a sign or swap slip in one of the two
fails); and, as Sec. II states for every choice of f^12, f^15, f^16, the
scheme's hydrodynamic modes agree with version 1's up to third order in k.
Versions 1 and 3 are pinned (version 3 against the discrete Maxwellian's
moments).
"""
import numpy as np

from . import d2v16

R_GAS = 1.0


def conserved(f, M=None):
    """(rho, jx, jy, e) = rows 1-4 of M applied to f (f has q as axis 0)."""
    if M is None:
        M = d2v16.moment_matrix()
    fh = np.tensordot(M[:4], f, axes=(1, 0))
    return fh[0], fh[1], fh[2], fh[3]


def primitive(rho, jx, jy, e):
    """u = j / rho and T from e = rho (T + u^2 / 2), R = 1 (Sec. II)."""
    ux = jx / rho
    uy = jy / rho
    T = (e / rho - 0.5 * (ux * ux + uy * uy)) / R_GAS
    return ux, uy, T


def feq_hat(rho, jx, jy, e, version=1):
    """Equilibrium moments f^eq_1..16, stacked on a new axis 0.

    Written in the paper's variables (Eqs. 14a-14i), with T from
    ``primitive`` where the version needs it.
    """
    if version not in (1, 2, 3):
        raise ValueError("equilibrium version must be 1, 2 or 3")
    ux, uy, T = primitive(rho, jx, jy, e)
    jj = jx * jx + jy * jy
    out = [None] * 16
    out[0] = rho
    out[1] = jx
    out[2] = jy
    out[3] = e
    out[4] = (jx * jx - jy * jy) / rho                                  # 14a
    out[5] = jx * jy / rho                                              # 14b
    out[6] = (e + rho * R_GAS * T) * jx / rho                           # 14c
    out[7] = (e + rho * R_GAS * T) * jy / rho                           # 14d
    out[8] = (jx * jx - 3.0 * jy * jy) * jx / rho ** 2                  # 14e
    out[9] = (3.0 * jx * jx - jy * jy) * jy / rho ** 2                  # 14f
    out[10] = 2.0 * e * e / rho - jj * jj / (4.0 * rho ** 3)            # 14g
    out[12] = (6.0 * rho * e - 2.0 * jj) * (jx * jx - jy * jy) / rho ** 3  # 14h
    out[13] = (6.0 * rho * e - 2.0 * jj) * jx * jy / rho ** 3           # 14i
    zero = 0.0 * rho
    if version == 1:
        out[11] = zero
        out[14] = zero
        out[15] = zero
    elif version == 2:
        out[11] = zero
        out[14] = rho * ux * (-4.0 + 10.0 * T + 5.0 * ux * ux - 5.0 * uy * uy)
        out[15] = rho * uy * (4.0 - 10.0 * T + 5.0 * ux * ux - 5.0 * uy * uy)
    else:
        M = d2v16.moment_matrix()
        fmax = maxwellian_discrete(rho, ux, uy, T)
        for k in (11, 14, 15):
            out[k] = np.tensordot(M[k], fmax, axes=(0, 0))
    return np.stack(out)


def maxwellian_discrete(rho, ux, uy, T):
    """f_i^max = rho/(2 pi T) exp(-(v_i - u)^2 / (2T)) on the 16 velocities."""
    v = d2v16.velocities().astype(float)
    out = []
    for q in range(16):
        d2 = (v[q, 0] - ux) ** 2 + (v[q, 1] - uy) ** 2
        out.append(rho / (2.0 * np.pi * T) * np.exp(-d2 / (2.0 * T)))
    return np.stack(out)


def feq(rho, ux, uy, T, version=1, Minv=None):
    """Discrete equilibrium in velocity space, f^eq = M^-1 f^eq_hat."""
    if Minv is None:
        Minv = d2v16.moment_matrix_inverse()
    jx = rho * ux
    jy = rho * uy
    e = rho * (R_GAS * T + 0.5 * (ux * ux + uy * uy))
    return np.tensordot(Minv, feq_hat(rho, jx, jy, e, version), axes=(1, 0))
