"""Closed-form steady thermal Couette temperature profile (oracle).

TEST INFRASTRUCTURE ONLY.

Sec. IV A compares the simulated Couette temperature with

    T = T1 + (T2 - T1) x/H + (mu / (2 lambda)) U^2 (x/H) (1 - x/H).

For a channel whose walls are normal to y, with u = (u_x(y), 0), the
momentum equation keeps the pressure uniform, so mu = p/s and lambda =
2p/s' (Sec. II, after Eq. 15d) are constant and the profile is the exact
steady solution of the energy equation.  Which rates enter:

* modified model (Eq. 5): the y energy flux is lambda_2 dT/dy + mu_v u_x
  du_x/dy, with mu_v = rho T/s6 and lambda_2 = 2 rho T/s8, so the bump
  coefficient is mu_v / (2 lambda_2) = s8 / (4 s6) = Pr / 4.
* unmodified model (Eq. 15d): the same flux is lambda_2 (dT/dy +
  (1/2) u_x du_x/dy), whatever the rates: the bump coefficient is 1/4.
"""
import numpy as np


def bump_coefficient(s6, s8, modified=True):
    """mu / (2 lambda) of the closed form for walls normal to y."""
    return s8 / (4.0 * s6) if modified else 0.25


def temperature(y, T0, T1, U, s6, s8, modified=True):
    """Steady T at wall-normal coordinate y in [0, 1] (H = 1)."""
    y = np.asarray(y, dtype=float)
    return T0 + (T1 - T0) * y + bump_coefficient(s6, s8, modified) * U * U * y * (1.0 - y)


def velocity(y, U):
    """Steady u_x(y) = U y: the wall at y = 0 is at rest, the one at y = 1 moves at U."""
    return U * np.asarray(y, dtype=float)
