"""Pin of the modified energy-flux collision by thermal Couette flow (Sec. IV A).

The steady state of the oracle's discrete scheme is found directly by
Newton's method on F(f) = (step(f) - f) / dt with the complex-step Jacobian,
so the time step can be small enough that the Lax-Wendroff term (whose
artificial diffusion 1/2 dt v^2 shifts the transport coefficients by
O(s dt)) no longer matters.  Central differences couple a node to its
neighbours two cells away in the viscous and conductive terms, so in steady
state the nodes split into two sub-lattices; the one holding the walls is
fixed by the boundary data and is the one compared (the other one's level is
undetermined in the dt -> 0 limit and Newton takes the minimum-norm
correction for it).

Expected profiles (closed form of Sec. IV A, coefficient from Sec. II):
  modified:   T = T0 + (T1 - T0) y + (Pr/4) U^2 y (1 - y),  Pr = s8/s6
  unmodified: T = T0 + (T1 - T0) y + (1/4) U^2 y (1 - y) whatever Pr.
"""
import numpy as np
import pytest

from oracle import couette, fdlb
from oracle import equilibrium as eq

U = 0.8


def _steady(Pr, modified, ny=11, s_visc=100.0, s_other=1000.0, dt=1e-6, iters=10):
    s = np.full(16, s_other)
    s[:4] = 0
    s[4] = s[5] = s_visc
    s[6] = s[7] = Pr * s_visc
    dy = 1.0 / (ny - 1)
    sides = (fdlb.Side(), fdlb.Side(), fdlb.Side(fdlb.WALL, 0.0, 0.0, 1.0),
             fdlb.Side(fdlb.WALL, U, 0.0, 1.0))
    p = fdlb.Params(nx=1, ny=ny, dx=dy, dy=dy, dt=dt, s=s, sides=sides, modified=modified)
    y = np.arange(ny) * dy
    T = couette.temperature(y, 1.0, 1.0, U, s_visc, Pr * s_visc, modified)
    ux = couette.velocity(y, U)
    f = fdlb.prepare(eq.feq((1 / T)[:, None], ux[:, None], 0 * ux[:, None], T[:, None]), p)
    n = f.size
    for _ in range(iters):
        G = ((fdlb.step(f, p) - f) / dt).ravel()
        J = np.empty((n, n))
        for c in range(n):
            fc = f.astype(complex).ravel()
            fc[c] += 1e-30j
            J[:, c] = (fdlb.step(fc.reshape(f.shape), p).ravel().imag / 1e-30
                       - (np.arange(n) == c)) / dt
        d = np.linalg.lstsq(J, -G, rcond=1e-12)[0]
        f = f + d.reshape(f.shape)
    _, u, _, Tn = fdlb.macros(f)
    return y, u[:, 0], Tn[:, 0]


@pytest.mark.parametrize("Pr,modified", [(0.5, True), (2.0, True), (2.0, False), (0.5, False)])
def test_couette_steady_state_matches_closed_form(Pr, modified):
    y, u, T = _steady(Pr, modified)
    s6, s8 = 100.0, 100.0 * Pr
    T_ref = couette.temperature(y, 1.0, 1.0, U, s6, s8, modified)
    bump = couette.bump_coefficient(s6, s8, modified) * U * U / 4  # bump at y = 1/2
    even = slice(0, None, 2)  # the wall sub-lattice (walls at nodes 0 and 10)
    assert np.abs(T[even] - T_ref[even]).max() < 2e-3 * bump
    assert np.abs(u[even] - U * y[even]).max() < 1e-3 * U


def test_couette_modification_changes_the_profile():
    """At Pr = 2 the modified and unmodified bumps differ by a factor of two."""
    y, _, Tm = _steady(2.0, True)
    _, _, Tu = _steady(2.0, False)
    k = 4  # y = 0.4, on the wall sub-lattice
    assert np.isclose((Tm[k] - 1.0) / (Tu[k] - 1.0), 2.0, rtol=2e-3)
