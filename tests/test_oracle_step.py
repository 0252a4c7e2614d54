"""Pins of the oracle's time step (Sec. II-III).

* brute force: an independent loop-per-node implementation on tiny grids,
  using the printed M (golden fixture) and a linear solve for M^-1;
* the amplification matrix G(k) printed in Sec. III (including the rows for
  the modified energy-flux collision) against the oracle's exact Jacobian
  (complex step) on a periodic grid around a uniform moving state;
* exact conservation of mass, momentum and energy on periodic grids;
* second-order convergence of the Lax-Wendroff advection with collision off;
* the complex-step tangent against central finite differences.
"""
import os

import numpy as np
import pytest

from oracle import d2v16, fdlb
from oracle.stability import amplification_matrix
from oracle import equilibrium as eq

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _printed_M():
    from fractions import Fraction
    rows = []
    with open(os.path.join(GOLDEN, "paper_M_rows.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append([float(Fraction(t)) for t in line.split()])
    return np.array(rows)


# ---------------------------------------------------------------------------
# brute force
# ---------------------------------------------------------------------------
def _macros_by_sums(g, v):
    rho = g.sum()
    jx = (g * v[:, 0]).sum()
    jy = (g * v[:, 1]).sum()
    e = (g * 0.5 * (v ** 2).sum(1)).sum()
    return rho, jx, jy, e


def _feq_solve(Mp, rho, ux, uy, T, version):
    e = rho * (T + 0.5 * (ux * ux + uy * uy))
    return np.linalg.solve(Mp, eq.feq_hat(rho, rho * ux, rho * uy, e, version))


def brute_step(f, p):
    Mp = _printed_M()
    v = d2v16.velocities().astype(float)
    nq, ny, nx = f.shape
    kinds = [s.kind for s in p.sides]
    f = f.copy()

    def nee(fr):
        out = fr.copy()
        for side, (wi, wj, ai, aj) in enumerate(
                [(lambda k: 0, lambda k: k, lambda k: 1, lambda k: k),
                 (lambda k: nx - 1, lambda k: k, lambda k: nx - 2, lambda k: k),
                 (lambda k: k, lambda k: 0, lambda k: k, lambda k: 1),
                 (lambda k: k, lambda k: ny - 1, lambda k: k, lambda k: ny - 2)]):
            if kinds[side] != fdlb.WALL:
                continue
            n = ny if side < 2 else nx
            sd = p.sides[side]
            for k in range(n):
                ga = fr[:, aj(k), ai(k)]
                rho, jx, jy, e = _macros_by_sums(ga, v)
                ux, uy = jx / rho, jy / rho
                T = e / rho - 0.5 * (ux * ux + uy * uy)
                out[:, wj(k), wi(k)] = (_feq_solve(Mp, rho, sd.ux, sd.uy, sd.T, p.version)
                                        + ga - _feq_solve(Mp, rho, ux, uy, T, p.version))
        return out

    f = nee(f)

    def at(i, j):
        # ghost rule: periodic wraps, everything else copies the edge node
        if i < 0 or i >= nx:
            i = (i % nx) if kinds[0] == fdlb.PERIODIC else min(max(i, 0), nx - 1)
        if j < 0 or j >= ny:
            j = (j % ny) if kinds[2] == fdlb.PERIODIC else min(max(j, 0), ny - 1)
        return f[:, j, i]

    def vel(i, j):
        rho, jx, jy, e = _macros_by_sums(at(i, j), v)
        return jx / rho, jy / rho

    out = f.copy()
    s = p.s
    for j in range(ny):
        for i in range(nx):
            if (kinds[0] == fdlb.WALL and i == 0) or (kinds[1] == fdlb.WALL and i == nx - 1) \
                    or (kinds[2] == fdlb.WALL and j == 0) or (kinds[3] == fdlb.WALL and j == ny - 1):
                continue
            g = at(i, j)
            rho, jx, jy, e = _macros_by_sums(g, v)
            ux, uy = jx / rho, jy / rho
            T = e / rho - 0.5 * (ux * ux + uy * uy)
            fh = Mp @ g
            fe = eq.feq_hat(rho, jx, jy, e, p.version)
            c = np.zeros(16)
            for k in range(4, 16):
                c[k] = s[k] * (fh[k] - fe[k])
            if p.modified:
                uE, uW, uN, uS = vel(i + 1, j), vel(i - 1, j), vel(i, j + 1), vel(i, j - 1)
                dxux = (uE[0] - uW[0]) / (2 * p.dx)
                dxuy = (uE[1] - uW[1]) / (2 * p.dx)
                dyux = (uN[0] - uS[0]) / (2 * p.dy)
                dyuy = (uN[1] - uS[1]) / (2 * p.dy)
                c[6] += (s[6] / s[4] - 1) * rho * T * ux * (dxux - dyuy) \
                    + (s[6] / s[5] - 1) * rho * T * uy * (dxuy + dyux)
                c[7] += (s[7] / s[5] - 1) * rho * T * ux * (dxuy + dyux) \
                    + (s[7] / s[4] - 1) * rho * T * uy * (dxux - dyuy)
            C = np.linalg.solve(Mp, c)
            for q in range(16):
                adv = 0.0
                for a, (di, dj), d in ((0, (1, 0), p.dx), (1, (0, 1), p.dy)):
                    if v[q, a] == 0:
                        continue
                    fp = at(i + di, j + dj)[q]
                    fm = at(i - di, j - dj)[q]
                    nu = v[q, a] * p.dt / d
                    adv += 0.5 * nu * (fp - fm) - 0.5 * nu * nu * (fp - 2 * g[q] + fm)
                out[q, j, i] = g[q] - adv - p.dt * C[q]
    return nee(out)


def _near_eq(nx, ny, seed, amp=1e-3):
    rng = np.random.default_rng(seed)
    rho = 1.0 + 0.2 * rng.uniform(-1, 1, (ny, nx))
    ux = 0.3 * rng.uniform(-1, 1, (ny, nx))
    uy = 0.3 * rng.uniform(-1, 1, (ny, nx))
    T = 1.0 + 0.2 * rng.uniform(-1, 1, (ny, nx))
    return eq.feq(rho, ux, uy, T) + amp * rng.standard_normal((16, ny, nx))


def _rates(seed):
    s = np.random.default_rng(seed).uniform(50, 400, 16)
    s[:4] = 0
    return s


SIDE_SETS = {
    "periodic": (fdlb.Side(), fdlb.Side(), fdlb.Side(), fdlb.Side()),
    "outflow_x": (fdlb.Side(fdlb.OUTFLOW), fdlb.Side(fdlb.OUTFLOW), fdlb.Side(), fdlb.Side()),
    "outflow_xy": (fdlb.Side(fdlb.OUTFLOW),) * 4,
    "walls_y": (fdlb.Side(), fdlb.Side(), fdlb.Side(fdlb.WALL, 0.1, 0.0, 1.1),
                fdlb.Side(fdlb.WALL, 0.5, -0.05, 0.95)),
    "walls_x": (fdlb.Side(fdlb.WALL, 0.02, 0.3, 1.0), fdlb.Side(fdlb.WALL, 0.0, -0.2, 1.2),
                fdlb.Side(fdlb.OUTFLOW), fdlb.Side(fdlb.OUTFLOW)),
}


@pytest.mark.parametrize("sides", list(SIDE_SETS))
@pytest.mark.parametrize("version", [1, 3])
def test_step_matches_brute_force(sides, version):
    nx, ny = 5, 4
    p = fdlb.Params(nx=nx, ny=ny, dx=0.1, dy=0.07, dt=2e-3, s=_rates(11),
                    sides=SIDE_SETS[sides], version=version, modified=True)
    f = fdlb.prepare(_near_eq(nx, ny, 12), p)
    a = fdlb.step(f, p)
    b = brute_step(f, p)
    assert np.abs(a - b).max() < 1e-13 * np.abs(b).max()


# ---------------------------------------------------------------------------
# amplification matrix G(k) of Sec. III
# ---------------------------------------------------------------------------
def _jacobian(p, f0):
    n = f0.size
    J = np.empty((n, n))
    h = 1e-30
    for c in range(n):
        fc = f0.astype(complex).ravel()
        fc[c] += 1j * h
        J[:, c] = fdlb.step(fc.reshape(f0.shape), p).ravel().imag / h
    return J


@pytest.mark.parametrize("modified", [True, False])
def test_linearised_step_is_papers_amplification_matrix(modified):
    nx, ny = 6, 5
    s = np.array([0, 0, 0, 0, 1e4, 2e4, 3e4, 5e3, 1e5, 5e4, 2e4, 8e4, 1.5e4, 6e4, 3e4, 9e4])
    p = fdlb.Params(nx=nx, ny=ny, dx=1e-3, dy=1.3e-3, dt=1e-5, s=s, modified=modified)
    rho, ux, uy, T = 2.0, 2.0, -0.7, 2.0
    f0 = eq.feq(np.full((ny, nx), rho), np.full((ny, nx), ux), np.full((ny, nx), uy),
                np.full((ny, nx), T))
    J = _jacobian(p, f0).reshape(16, ny, nx, 16, ny, nx)
    for mx, my in ((1, 0), (0, 2), (2, 1), (3, 2)):
        kx = 2 * np.pi * mx / (nx * p.dx)
        ky = 2 * np.pi * my / (ny * p.dy)
        ph = np.exp(1j * (kx * p.dx * np.arange(nx)[None, :] + ky * p.dy * np.arange(ny)[:, None]))
        Gnum = np.einsum("qpyx,yx->qp", J[:, 0, 0], ph)
        Gp = amplification_matrix(p, rho, ux, uy, T, kx, ky)
        assert np.abs(Gnum - Gp).max() < 1e-11, (mx, my, np.abs(Gnum - Gp).max())


# ---------------------------------------------------------------------------
# conservation, convergence, tangent
# ---------------------------------------------------------------------------
def test_periodic_step_conserves_totals():
    nx, ny = 8, 6
    p = fdlb.Params(nx=nx, ny=ny, dx=0.05, dy=0.05, dt=2e-3, s=_rates(21))
    f = _near_eq(nx, ny, 22, amp=1e-2)
    v = d2v16.velocities().astype(float)
    w = np.stack([np.ones(16), v[:, 0], v[:, 1], 0.5 * (v ** 2).sum(1)])
    before = np.einsum("kq,qyx->k", w, f)
    for _ in range(20):
        f = fdlb.step(f, p)
    after = np.einsum("kq,qyx->k", w, f)
    assert np.abs(after - before).max() < 1e-12 * np.abs(before).max()


def _advect_error(n, kx, ky):
    d = 1.0 / n
    dt = 0.2 * d  # Courant number 0.4 for speed 2
    p = fdlb.Params(nx=n, ny=n, dx=d, dy=d, dt=dt, s=np.zeros(16), modified=False)
    x = (np.arange(n) + 0.5) * d
    X, Y = np.meshgrid(x, x)
    v = d2v16.velocities().astype(float)
    f = np.stack([1.0 + 0.1 * np.sin(2 * np.pi * (kx * X + ky * Y)) for _ in range(16)])
    nsteps = int(round(0.1 / dt))
    for _ in range(nsteps):
        f = fdlb.step(f, p)
    t = nsteps * dt
    exact = np.stack([1.0 + 0.1 * np.sin(2 * np.pi * (kx * (X - v[q, 0] * t) + ky * (Y - v[q, 1] * t)))
                      for q in range(16)])
    return np.abs(f - exact).max(axis=(1, 2))


def test_lax_wendroff_second_order_along_one_axis():
    """Collision off, a wave along x: every f_i is advected by the 1D
    Lax-Wendroff scheme and the error drops ~4x per refinement."""
    e1, e2 = _advect_error(24, 1, 0), _advect_error(48, 1, 0)
    moving = np.abs(d2v16.velocities()[:, 0]) > 0
    ratio = e1[moving] / e2[moving]
    assert (ratio > 3.3).all() and (ratio < 4.7).all(), ratio


def test_axis_split_scheme_has_no_cross_term():
    """G of Sec. III carries (v_a dt / dx_a)^2 per axis and no x-y cross term,
    so for a wave varying along x and y the diagonal velocities keep the
    first-order forward-Euler error dt v_x v_y d2f/dxdy: their error halves
    under refinement, while the axis velocities stay second order."""
    e1, e2 = _advect_error(24, 1, 2), _advect_error(48, 1, 2)
    v = d2v16.velocities()
    diag = (v[:, 0] != 0) & (v[:, 1] != 0)
    ratio = e1 / e2
    assert (ratio[diag] > 1.7).all() and (ratio[diag] < 2.5).all(), ratio
    assert (ratio[~diag] > 3.3).all(), ratio


def test_complex_step_tangent_matches_finite_differences():
    nx, ny = 5, 4
    p = fdlb.Params(nx=nx, ny=ny, dx=0.05, dy=0.05, dt=1e-3, s=_rates(31),
                    sides=SIDE_SETS["walls_y"])
    f = fdlb.prepare(_near_eq(nx, ny, 32), p)
    w = np.random.default_rng(33).standard_normal(f.shape)
    h = 1e-30
    tan = fdlb.step(f + 1j * h * w, p).imag / h
    eps = 1e-6
    fd = (fdlb.step(f + eps * w, p) - fdlb.step(f - eps * w, p)) / (2 * eps)
    assert np.abs(tan - fd).max() < 1e-7 * np.abs(tan).max()
