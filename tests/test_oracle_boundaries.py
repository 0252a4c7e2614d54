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
