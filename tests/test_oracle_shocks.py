"""Pins of the shocked-flow references (Sec. III, IV B) and of the oracle's
step against the exact Riemann solution.

gamma = 2 for the model's gas (R = 1, e = rho (T + u^2/2)) is pinned by the
Mach numbers the paper prints (Ma = u / sqrt(2T)) and by its Mach-1.22
post-shock state; the exact solver is pinned by the jump conditions it must
satisfy and by the classical gamma = 1.4 Sod values (Toro, Riemann Solvers
and Numerical Methods for Fluid Dynamics, Table 4.3, test 1).
"""
import math
import os

import numpy as np
import pytest

from oracle import equilibrium as eq
from oracle import fdlb, riemann

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                key, *vals = line.split()
                out[key] = [float(v) for v in vals]
    return out


def test_printed_mach_numbers_fix_gamma_two():
    rows = np.loadtxt(os.path.join(GOLDEN, "paper_mach_numbers.txt"))
    for u, T, ma, digits in rows:
        c = math.sqrt(riemann.GAMMA * T)  # sound speed sqrt(gamma p / rho), p = rho T
        assert round(u / c, int(digits)) == ma


def test_printed_shock_bubble_state_is_rankine_hugoniot_gamma_two():
    g = _golden("paper_shock_bubble.txt")
    rho1, u1, _, p1 = g["pre_shock"]
    rho2, u2, p2, D = riemann.shock_state(rho1, p1, g["mach"][0], direction=-1)
    assert round(D, 3) == g["D"][0]
    r, u, _, p = g["post_shock"]
    assert round(rho2, 2) == r
    assert round(u2, 4) == u
    assert round(p2, 4) == p
    # the bubble sits at the pre-shock pressure
    assert g["bubble"][3] == p1


@pytest.mark.parametrize("mach", [1.22, 1.5, 3.0, 10.0])
def test_shock_state_satisfies_jump_conditions(mach):
    g = riemann.GAMMA
    rho2, u2, p2, D = riemann.shock_state(1.0, 1.0, mach)
    w1, w2 = D, D - u2  # shock-frame speeds
    E = lambda rho, w, p: 0.5 * rho * w * w + p / (g - 1)
    assert np.isclose(1.0 * w1, rho2 * w2, rtol=1e-12)
    assert np.isclose(1.0 + 1.0 * w1 * w1, p2 + rho2 * w2 * w2, rtol=1e-12)
    assert np.isclose((E(1.0, w1, 1.0) + 1.0) * w1, (E(rho2, w2, p2) + p2) * w2, rtol=1e-12)
    assert rho2 > 1.0 and p2 > 1.0  # compressive


def test_exact_solver_reproduces_textbook_sod_gamma_14():
    ps, us = riemann.star_state((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), g=1.4)
    assert round(ps, 5) == 0.30313
    assert round(us, 5) == 0.92745


def test_exact_solution_structure_gamma_two():
    left, right = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)
    ps, us = riemann.star_state(left, right)
    xi = np.linspace(-3, 3, 6001)
    rho, u, p = riemann.exact_riemann(left, right, xi)
    # far states
    assert (rho[0], u[0], p[0]) == left and (rho[-1], u[-1], p[-1]) == right
    # p and u continuous across the contact (both equal the star values there)
    star = (xi > us - 0.2) & (xi < us + 0.2)
    assert np.allclose(p[star], ps) and np.allclose(u[star], us)
    # left rarefaction: isentropic, p / rho^gamma constant through the fan
    fan = (xi > -math.sqrt(2.0)) & (xi < us - 0.3)
    assert np.allclose(p[fan] / rho[fan] ** 2, 1.0, rtol=1e-12)
    # right shock: Rankine-Hugoniot between the star-right and right states
    g = 2.0
    rs = rho[np.searchsorted(xi, us + 0.1)]
    mu = (g - 1) / (g + 1)
    assert np.isclose(rs, right[0] * (ps / right[2] + mu) / (mu * ps / right[2] + 1), rtol=1e-12)


def _sod(nx, nsteps=1500, dt=1e-5):
    s = np.full(16, 1e5)
    s[:4] = 0
    s[4:8] = 1.5e4
    dx = 1.0 / nx
    p = fdlb.Params(nx=nx, ny=1, dx=dx, dy=dx, dt=dt, s=s,
                    sides=(fdlb.Side(fdlb.OUTFLOW), fdlb.Side(fdlb.OUTFLOW), fdlb.Side(), fdlb.Side()))
    x = (np.arange(nx) + 0.5) * dx
    w = 0.5 * (1 + np.tanh((x - 0.5) / (2 * dx)))
    rho = 1 + (0.125 - 1) * w
    T = 1 + (0.8 - 1) * w
    f = eq.feq(rho[None], 0 * rho[None], 0 * rho[None], T[None])
    f = fdlb.run(f, p, nsteps)
    r, u, _, Tn = fdlb.macros(f)
    re, ue, pe = riemann.exact_riemann((1, 0, 1), (0.125, 0, 0.1), (x - 0.5) / (nsteps * dt))
    return np.abs(r[0] - re).mean(), np.abs(u[0] - ue).mean(), np.abs(r[0] * Tn[0] - pe).mean()


def test_oracle_sod_tube_approaches_exact_solution():
    """Sod tube (rho, T) = (1, 1) | (0.125, 0.8) at t = 0.015: the L1 error
    against the gamma = 2 exact solution is small and shrinks under
    refinement at a fixed smoothing of 2 cells."""
    e400 = _sod(400)
    e800 = _sod(800)
    assert e400[0] < 4e-3 and e400[1] < 1e-2 and e400[2] < 4e-3
    assert all(b < 0.8 * a for a, b in zip(e400, e800)), (e400, e800)
