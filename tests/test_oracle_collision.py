"""Pins of the collision (Eq. 3 with the Sec. II modification)."""
import numpy as np
import pytest

from oracle import d2v16, fdlb
from oracle import equilibrium as eq


def _params(s, modified=True, version=1):
    return fdlb.Params(nx=1, ny=1, dx=1.0, dy=1.0, dt=1.0, s=s, modified=modified, version=version)


def _random_state(seed, n=50):
    rng = np.random.default_rng(seed)
    f = rng.uniform(0.02, 0.2, size=(16, n))
    grad = tuple(rng.normal(size=n) for _ in range(4))
    rho, jx, jy, e = eq.conserved(f)
    return f, rho, jx, jy, e, grad


def _rates(seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(1e2, 1e4, size=16)


@pytest.mark.parametrize("version", [1, 2, 3])
@pytest.mark.parametrize("modified", [True, False])
def test_collision_conserves_mass_momentum_energy(version, modified):
    f, rho, jx, jy, e, grad = _random_state(1)
    C = fdlb.collision(f, rho, jx, jy, e, grad, _params(_rates(2), modified, version))
    v = d2v16.velocities().astype(float)
    scale = np.abs(C).max()
    assert np.abs(C.sum(0)).max() < 1e-13 * scale
    assert np.abs((C * v[:, 0:1]).sum(0)).max() < 1e-13 * scale
    assert np.abs((C * v[:, 1:2]).sum(0)).max() < 1e-13 * scale
    assert np.abs((C * 0.5 * (v ** 2).sum(1)[:, None]).sum(0)).max() < 1e-13 * scale


@pytest.mark.parametrize("version", [1, 2, 3])
def test_collision_vanishes_at_equilibrium_without_gradients(version):
    rho, ux, uy, T = np.array([1.3, 0.2]), np.array([0.4, -1.0]), np.array([-0.7, 0.1]), np.array([0.9, 2.0])
    f = eq.feq(rho, ux, uy, T, version)
    r, jx, jy, e = eq.conserved(f)
    zero = np.zeros(2)
    C = fdlb.collision(f, r, jx, jy, e, (zero,) * 4, _params(_rates(3), True, version))
    assert np.abs(C).max() < 1e-10 * np.abs(f).max() * _rates(3).max()


def test_single_relaxation_limit():
    """All s_k = s, unmodified: the MRT operator is s (f - f^eq) (Sec. II)."""
    f, rho, jx, jy, e, grad = _random_state(4)
    s = 1234.5
    C = fdlb.collision(f, rho, jx, jy, e, grad, _params(np.full(16, s), modified=False))
    ux, uy, T = eq.primitive(rho, jx, jy, e)
    ref = s * (f - eq.feq(rho, ux, uy, T, 1))
    assert np.allclose(C, ref, rtol=1e-11, atol=1e-11 * np.abs(ref).max())


def test_conserved_rates_have_no_effect():
    f, rho, jx, jy, e, grad = _random_state(5)
    s = _rates(6)
    C1 = fdlb.collision(f, rho, jx, jy, e, grad, _params(s))
    s2 = s.copy()
    s2[:4] = [7.0, -3.0, 1e9, 0.5]
    C2 = fdlb.collision(f, rho, jx, jy, e, grad, _params(s2))
    assert np.array_equal(C1, C2)


def test_modification_vanishes_at_unit_prandtl():
    """s5 = s6 = s7 = s8: every (s_a/s_b - 1) factor is zero."""
    f, rho, jx, jy, e, grad = _random_state(7)
    s = _rates(8)
    s[4:8] = 2500.0
    Cm = fdlb.collision(f, rho, jx, jy, e, grad, _params(s, modified=True))
    Cu = fdlb.collision(f, rho, jx, jy, e, grad, _params(s, modified=False))
    assert np.array_equal(Cm, Cu)


def test_modification_only_touches_energy_flux_moments():
    """The modification changes moments 7 and 8 of M C only (Sec. II)."""
    f, rho, jx, jy, e, grad = _random_state(9)
    s = _rates(10)
    M = d2v16.moment_matrix()
    Cm = fdlb.collision(f, rho, jx, jy, e, grad, _params(s, True))
    Cu = fdlb.collision(f, rho, jx, jy, e, grad, _params(s, False))
    dm = M @ (Cm - Cu)
    scale = np.abs(M @ Cu).max()
    others = [k for k in range(16) if k not in (6, 7)]
    assert np.abs(dm[others]).max() < 1e-13 * scale
    assert np.abs(dm[6]).max() > 0 and np.abs(dm[7]).max() > 0
