"""Pins of the oracle's inflow and reflecting boundaries (Sec. IV B).

Reflection: the lattice, M, the equilibria and the modification are all
symmetric under a mirror across an axis, so a run with reflecting sides
equals the matching half of a periodic run on the mirror-doubled domain.
Inflow: a uniform state equal to the inflow state is a steady solution.
"""
import numpy as np

from oracle import d2v16
from oracle import equilibrium as oeq
from oracle import fdlb


def _smooth_state(nx, ny, seed):
    rng = np.random.default_rng(seed)
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    X, Y = np.meshgrid(x, y)
    a = rng.uniform(-1, 1, 6)
    rho = 1.0 + 0.1 * np.sin(2 * np.pi * X + a[0]) * np.cos(2 * np.pi * Y + a[1])
    ux = 0.1 * np.cos(2 * np.pi * Y + a[2]) + 0.05 * np.sin(2 * np.pi * X)
    uy = 0.08 * np.sin(2 * np.pi * X + a[3]) * np.sin(np.pi * Y + a[4])
    T = 1.0 + 0.05 * np.cos(2 * np.pi * X + a[5])
    f = oeq.feq(rho, ux, uy, T) + 1e-3 * rng.standard_normal((16, ny, nx))
    return f


def _params(nx, ny, sides):
    s = np.random.default_rng(3).uniform(100, 2000, 16)
    s[:4] = 0
    return fdlb.Params(nx=nx, ny=ny, dx=0.01, dy=0.012, dt=2e-4, s=s, sides=sides)


def test_mirror_permutations_negate_one_component():
    v = d2v16.velocities()
    for axis in (0, 1):
        p = fdlb.mirror_permutation(axis)
        w = v.copy()
        w[:, axis] *= -1
        assert np.array_equal(v[p], w)
        assert np.array_equal(p[p], np.arange(16))


def test_reflect_in_y_equals_mirror_doubled_periodic_run():
    nx, ny, K = 10, 7, 6
    f = _smooth_state(nx, ny, 1)
    per = fdlb.Side(fdlb.PERIODIC)
    ref = fdlb.Side(fdlb.REFLECT)
    got = fdlb.run(f, _params(nx, ny, (per, per, ref, ref)), K)
    # rows ny..2ny-1 of the doubled domain: row ny + k = mirror of row ny - 1 - k
    m = fdlb.mirror_permutation(1)
    big = np.concatenate([f, f[m][:, ::-1, :]], axis=1)
    want = fdlb.run(big, _params(nx, 2 * ny, (per, per, per, per)), K)[:, :ny, :]
    assert np.abs(got - want).max() < 1e-13 * np.abs(want).max()


def test_reflect_in_x_equals_mirror_doubled_periodic_run():
    nx, ny, K = 8, 9, 6
    f = _smooth_state(nx, ny, 2)
    per = fdlb.Side(fdlb.PERIODIC)
    ref = fdlb.Side(fdlb.REFLECT)
    got = fdlb.run(f, _params(nx, ny, (ref, ref, per, per)), K)
    m = fdlb.mirror_permutation(0)
    big = np.concatenate([f, f[m][:, :, ::-1]], axis=2)
    want = fdlb.run(big, _params(2 * nx, ny, (per, per, per, per)), K)[:, :, :nx]
    assert np.abs(got - want).max() < 1e-13 * np.abs(want).max()


def test_uniform_inflow_state_is_steady():
    nx, ny = 12, 5
    state = dict(rho=1.28, ux=-0.3774, uy=0.0, T=1.6512 / 1.28)
    inflow = fdlb.Side(fdlb.INFLOW, ux=state["ux"], uy=state["uy"], T=state["T"], rho=state["rho"])
    p = _params(nx, ny, (fdlb.Side(fdlb.OUTFLOW), inflow, fdlb.Side(fdlb.REFLECT), fdlb.Side(fdlb.REFLECT)))
    one = np.ones((ny, nx))
    f0 = oeq.feq(state["rho"] * one, state["ux"] * one, state["uy"] * one, state["T"] * one)
    f = fdlb.run(f0, p, 10)
    assert np.abs(f - f0).max() < 1e-14 * np.abs(f0).max()


def test_inflow_ghost_is_the_side_equilibrium():
    nx, ny = 6, 4
    inflow = fdlb.Side(fdlb.INFLOW, ux=0.3, uy=-0.1, T=0.9, rho=2.0)
    p = _params(nx, ny, (inflow, fdlb.Side(fdlb.OUTFLOW), fdlb.Side(fdlb.PERIODIC), fdlb.Side(fdlb.PERIODIC)))
    g = fdlb._ghosts(_smooth_state(nx, ny, 4), p)
    want = oeq.feq(np.array([2.0]), np.array([0.3]), np.array([-0.1]), np.array([0.9]))[:, 0]
    assert np.allclose(g[:, 1:-1, 0], want[:, None], rtol=0, atol=1e-15)


# ---------------------------------------------------------------------------
# diffuse reflection (Sec. IV A)
# ---------------------------------------------------------------------------
def test_diffuse_wall_keeps_a_resting_equilibrium():
    nx, ny = 6, 7
    dif = fdlb.Side(fdlb.DIFFUSE, 0.0, 0.0, 1.2)
    per = fdlb.Side(fdlb.PERIODIC)
    p = _params(nx, ny, (per, per, dif, dif))
    one = np.ones((ny, nx))
    f0 = oeq.feq(1.3 * one, 0 * one, 0 * one, 1.2 * one)
    f = fdlb.run(f0, p, 10)
    assert np.abs(f - f0).max() < 1e-14 * np.abs(f0).max()


def test_diffuse_walls_keep_the_total_mass():
    """rho_w is chosen so that the Lax-Wendroff update moves no mass across
    the wall: the total mass is exact while momentum and energy are not."""
    for sides in ((fdlb.Side(), fdlb.Side(), fdlb.Side(fdlb.DIFFUSE, -0.2, 0.05, 1.0),
                   fdlb.Side(fdlb.DIFFUSE, 0.2, 0.0, 1.1)),
                  (fdlb.Side(fdlb.DIFFUSE, 0.0, -0.2, 0.9), fdlb.Side(fdlb.DIFFUSE, 0.0, 0.2, 1.0),
                   fdlb.Side(), fdlb.Side())):
        nx, ny = 9, 8
        f = _smooth_state(nx, ny, 6)
        p = _params(nx, ny, sides)
        m0 = oeq.conserved(f)[0].sum()
        g = fdlb.run(f, p, 20)
        r, jx, jy, e = oeq.conserved(g)
        assert abs(r.sum() - m0) < 1e-13 * m0
        assert abs(e.sum() - oeq.conserved(f)[3].sum()) > 1e-10  # the walls exchange energy


def _slip_couette_steady(ny=12, U=0.2, s_visc=100.0, dt=1e-6, iters=8):
    """Newton on F(f) = (step(f) - f)/dt (complex-step Jacobian) for a
    channel between diffuse walls normal to y moving at -U and +U."""
    s = np.full(16, s_visc)
    s[:4] = 0
    d = 1.0 / ny
    sides = (fdlb.Side(), fdlb.Side(), fdlb.Side(fdlb.DIFFUSE, -U, 0.0, 1.0), fdlb.Side(fdlb.DIFFUSE, U, 0.0, 1.0))
    p = fdlb.Params(nx=1, ny=ny, dx=d, dy=d, dt=dt, s=s, sides=sides)
    y = (np.arange(ny) + 0.5) * d
    ux = U * (2 * y - 1)
    one = np.ones_like(y)
    f = oeq.feq(one[:, None], ux[:, None], 0 * ux[:, None], one[:, None])
    n = f.size
    for _ in range(iters):
        G = ((fdlb.step(f, p) - f) / dt).ravel()
        J = np.empty((n, n))
        for c in range(n):
            fc = f.astype(complex).ravel()
            fc[c] += 1e-30j
            J[:, c] = (fdlb.step(fc.reshape(f.shape), p).ravel().imag / 1e-30 - (np.arange(n) == c)) / dt
        f = f + np.linalg.lstsq(J, -G, rcond=1e-12)[0].reshape(f.shape)
    assert np.abs((fdlb.step(f, p) - f) / dt).max() < 1e-6
    _, u, _, T = fdlb.macros(f)
    return y, u[:, 0], T[:, 0]


def test_diffuse_slip_couette_shows_slip_and_a_temperature_jump():
    """Sec. IV A: with diffuse walls the fluid next to a wall lags the wall
    (velocity slip) and is hotter than it (temperature jump, from viscous
    heating); the profile is odd in u and even in T about the midline."""
    y, u, T = _slip_couette_steady()
    U = 0.2
    assert 0 < u[-1] < U and -U < u[0] < 0            # slip at both walls
    assert T[0] > 1.0 and T[-1] > 1.0                 # hotter than the walls
    assert T[len(T) // 2] > T[0]                      # heated in the middle
    assert np.allclose(u, -u[::-1], atol=1e-9) and np.allclose(T, T[::-1], atol=1e-9)
