"""Linear stability of the scheme (Sec. III): the amplification matrix G(k).

TEST INFRASTRUCTURE ONLY.

For a uniform state (rho, u, T) and a Fourier mode exp(i k.x), one step
maps f' to G(k) f'.  G is written out as Sec. III prints it: the diagonal
Lax-Wendroff symbol per velocity, minus dt M^-1 S (M - d f^eq/d f), with
the rows of moments 7 and 8 carrying the linearised modification (the
velocity derivatives in it take the central-difference symbol
i sin(k d)/d).  The scheme is stable for the state when every eigenvalue
of G(k) has modulus at most 1 for every k.  The oracle's own Jacobian of
fdlb.step equals this G to rounding (pinned in the tests).
"""
import numpy as np

from . import d2v16
from . import equilibrium as eq


def amplification_matrix(p, rho, ux, uy, T, kx, ky):
    """G_ij as printed in Sec. III, with the rows for moments 7 and 8 replaced
    as for the modified collision; spatial derivatives of u in the
    modification carry the central-difference symbol i sin(k d)/d."""
    M = d2v16.moment_matrix()
    Minv = d2v16.moment_matrix_inverse()
    v = d2v16.velocities().astype(float)
    s = p.s
    G = np.zeros((16, 16), dtype=complex)
    for i in range(16):
        adv = 0.0
        for a, k, d in ((0, kx, p.dx), (1, ky, p.dy)):
            nu = v[i, a] * p.dt / d
            adv += -nu / 2 * (np.exp(1j * k * d) - np.exp(-1j * k * d)) \
                + 0.5 * nu ** 2 * (np.exp(1j * k * d) - 2 + np.exp(-1j * k * d))
        G[i, i] = 1.0 + adv
    # d f^eq_k / d f_j through (rho, j, e), by complex step on the equilibrium
    f0 = eq.feq(np.array(rho), np.array(ux), np.array(uy), np.array(T))
    Deq = np.zeros((16, 16))
    for j in range(16):
        fc = f0.astype(complex)
        fc[j] += 1e-30j
        r, jx, jy, e = eq.conserved(fc)
        Deq[:, j] = eq.feq_hat(r, jx, jy, e, p.version).imag / 1e-30
    S = np.diag(s)
    G -= p.dt * Minv @ S @ (M - Deq)
    if p.modified:
        dux = (v[:, 0] - ux) / rho  # d u_x / d f_j
        duy = (v[:, 1] - uy) / rho
        Kx = 1j * np.sin(kx * p.dx) / p.dx
        Ky = 1j * np.sin(ky * p.dy) / p.dy
        rT = rho * T
        d7 = (s[6] / s[4] - 1) * rT * ux * (Kx * dux - Ky * duy) \
            + (s[6] / s[5] - 1) * rT * uy * (Kx * duy + Ky * dux)
        d8 = (s[7] / s[5] - 1) * rT * ux * (Kx * duy + Ky * dux) \
            + (s[7] / s[4] - 1) * rT * uy * (Kx * dux - Ky * duy)
        G -= p.dt * (np.outer(Minv[:, 6], d7) + np.outer(Minv[:, 7], d8))
    return G


def max_growth(p, rho, ux, uy, T, kdx, axis=0):
    """max over k d (array) of the largest eigenvalue modulus of G(k) along one axis."""
    d = p.dx if axis == 0 else p.dy
    out = 0.0
    for kd in np.asarray(kdx, dtype=float):
        k = kd / d
        G = amplification_matrix(p, rho, ux, uy, T, k if axis == 0 else 0.0, k if axis == 1 else 0.0)
        out = max(out, np.abs(np.linalg.eigvals(G)).max())
    return out
