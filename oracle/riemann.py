"""Exact Riemann solver and normal-shock states for an ideal gas (oracle).

TEST INFRASTRUCTURE ONLY.

The model's fluid is a 2D monatomic ideal gas with R = 1 (Sec. IV):
e = rho (T + u^2/2) means c_v = R = 1, c_p = 2, so gamma = 2 and
p = rho T.  The Mach numbers the paper quotes, Ma = u / sqrt(2 T)
(Sec. III, Sec. IV B), are u / sqrt(gamma p / rho) with gamma = 2, and its
Mach-1.22 post-shock state (Sec. IV B, Eq. of the bubble set-up) follows
from the jump conditions with gamma = 2.

``exact_riemann`` is the classical exact solver for the 1D Euler Riemann
problem (two-shock / two-rarefaction pressure function solved by Newton for
the star pressure, then sampled along x/t), written from the standard
textbook construction (Toro, "Riemann Solvers and Numerical Methods for
Fluid Dynamics", ch. 4).  ``shock_state`` solves the three Rankine-Hugoniot
jump conditions (mass, momentum, total enthalpy in the shock frame)
numerically, without the closed-form Mach relations.
"""
import math

import numpy as np
from scipy.optimize import brentq

GAMMA = 2.0


def _pressure_fn(p, rho_k, p_k, c_k, g=GAMMA):
    """Velocity jump across the left/right wave as a function of p*, and its derivative."""
    if p > p_k:  # shock
        a = 2.0 / ((g + 1.0) * rho_k)
        b = (g - 1.0) / (g + 1.0) * p_k
        sq = math.sqrt(a / (p + b))
        return (p - p_k) * sq, sq * (1.0 - 0.5 * (p - p_k) / (b + p))
    # rarefaction
    ex = (g - 1.0) / (2.0 * g)
    val = 2.0 * c_k / (g - 1.0) * ((p / p_k) ** ex - 1.0)
    der = 1.0 / (rho_k * c_k) * (p / p_k) ** (-(g + 1.0) / (2.0 * g))
    return val, der


def star_state(left, right, g=GAMMA, tol=1e-15):
    """(p*, u*) for primitive states left/right = (rho, u, p)."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl = math.sqrt(g * pl / rl)
    cr = math.sqrt(g * pr / rr)
    if 2.0 * (cl + cr) / (g - 1.0) <= ur - ul:
        raise ValueError("vacuum is generated")
    p = max(1e-12, 0.5 * (pl + pr))
    for _ in range(200):
        fl, dl = _pressure_fn(p, rl, pl, cl, g)
        fr, dr = _pressure_fn(p, rr, pr, cr, g)
        dp = (fl + fr + ur - ul) / (dl + dr)
        p_new = max(p - dp, 1e-14 * p)
        if abs(p_new - p) <= tol * 0.5 * (p_new + p):
            p = p_new
            break
        p = p_new
    fl, _ = _pressure_fn(p, rl, pl, cl, g)
    fr, _ = _pressure_fn(p, rr, pr, cr, g)
    return p, 0.5 * (ul + ur) + 0.5 * (fr - fl)


def exact_riemann(left, right, xi, g=GAMMA):
    """Sample the exact solution at similarity coordinates xi = (x - x0)/t.

    Returns arrays (rho, u, p) of xi's shape.
    """
    rl, ul, pl = left
    rr, ur, pr = right
    cl = math.sqrt(g * pl / rl)
    cr = math.sqrt(g * pr / rr)
    ps, us = star_state(left, right, g)
    xi = np.asarray(xi, dtype=float)
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    p = np.empty_like(xi)
    gm = (g - 1.0) / (g + 1.0)
    for n, s in np.ndenumerate(xi):
        if s <= us:  # left of the contact
            if ps > pl:  # left shock
                sl = ul - cl * math.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
                if s <= sl:
                    w = (rl, ul, pl)
                else:
                    w = (rl * (ps / pl + gm) / (gm * ps / pl + 1.0), us, ps)
            else:  # left rarefaction
                shl = ul - cl
                csl = cl * (ps / pl) ** ((g - 1) / (2 * g))
                stl = us - csl
                if s <= shl:
                    w = (rl, ul, pl)
                elif s >= stl:
                    w = (rl * (ps / pl) ** (1.0 / g), us, ps)
                else:
                    c = 2.0 / (g + 1) * (cl + (g - 1) / 2 * (ul - s))
                    uu = 2.0 / (g + 1) * (cl + (g - 1) / 2 * ul + s)
                    rr_ = rl * (c / cl) ** (2.0 / (g - 1))
                    w = (rr_, uu, pl * (c / cl) ** (2 * g / (g - 1)))
        else:  # right of the contact
            if ps > pr:  # right shock
                sr = ur + cr * math.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
                if s >= sr:
                    w = (rr, ur, pr)
                else:
                    w = (rr * (ps / pr + gm) / (gm * ps / pr + 1.0), us, ps)
            else:  # right rarefaction
                shr = ur + cr
                csr = cr * (ps / pr) ** ((g - 1) / (2 * g))
                str_ = us + csr
                if s >= shr:
                    w = (rr, ur, pr)
                elif s <= str_:
                    w = (rr * (ps / pr) ** (1.0 / g), us, ps)
                else:
                    c = 2.0 / (g + 1) * (cr - (g - 1) / 2 * (ur - s))
                    uu = 2.0 / (g + 1) * (-cr + (g - 1) / 2 * ur + s)
                    rr_ = rr * (c / cr) ** (2.0 / (g - 1))
                    w = (rr_, uu, pr * (c / cr) ** (2 * g / (g - 1)))
        rho[n], u[n], p[n] = w
    return rho, u, p


def shock_state(rho1, p1, mach, direction=+1, g=GAMMA):
    """Post-shock (rho2, u2, p2) behind a shock of Mach ``mach`` running into
    gas at rest (rho1, p1) in the +x (direction=+1) or -x direction.

    Solves the jump conditions in the shock frame:
      rho1 w1 = rho2 w2,  p1 + rho1 w1^2 = p2 + rho2 w2^2,
      g/(g-1) p1/rho1 + w1^2/2 = g/(g-1) p2/rho2 + w2^2/2,
    for the non-trivial root w2 < w1.  Returns also the shock speed D.
    """
    c1 = math.sqrt(g * p1 / rho1)
    D = mach * c1
    w1 = D
    m = rho1 * w1

    def energy_residual(w2):
        p2 = p1 + m * (w1 - w2)
        rho2 = m / w2
        return g / (g - 1) * (p2 / rho2 - p1 / rho1) + 0.5 * (w2 * w2 - w1 * w1)

    # the trivial root is w2 = w1; the physical one lies below the sonic speed
    w_lo = w1 * 1e-6
    w_hi = w1 * (1.0 - 1e-9)
    # bracket: scan for a sign change strictly below w1
    grid = np.linspace(w_lo, w_hi, 4001)
    vals = [energy_residual(w) for w in grid]
    k = next(i for i in range(len(grid) - 1) if vals[i] * vals[i + 1] < 0)
    w2 = brentq(energy_residual, grid[k], grid[k + 1], xtol=1e-15, rtol=1e-15)
    rho2 = m / w2
    p2 = p1 + m * (w1 - w2)
    u2 = direction * (w1 - w2)
    return rho2, u2, p2, D
