"""Pins of the equilibrium moments (Eqs. 14a-14i) against the Maxwellian.

The closed forms must equal the continuous 2D Maxwellian moments of each
row polynomial of M (Gauss-Hermite quadrature, exact for polynomials), and
the discrete equilibrium M^-1 f^eq must carry rho, j and e (Sec. II).
"""
import numpy as np
import pytest

from oracle import d2v16
from oracle import equilibrium as eq

STATES = [(1.0, 0.0, 0.0, 1.0), (1.3, 0.4, -0.7, 0.9), (0.125, 2.0, 1.0, 0.8),
          (5.0, 45.0, 0.0, 10.0), (3.0, -0.3, 0.5, 1.0 / 3.0)]


def _row_poly(k, a, b):
    v2 = a * a + b * b
    m9 = a ** 3 - 3 * a * b * b
    m10 = 3 * a * a * b - b ** 3
    return [1 + 0 * a, a, b, v2 / 2, a * a - b * b, a * b, v2 / 2 * a, v2 / 2 * b, m9, m10,
            v2 * v2 / 4, a ** 4 - 6 * a * a * b * b + b ** 4, v2 * (a * a - b * b), v2 * a * b,
            v2 * m9, v2 * m10][k]


def _maxwellian_moment(k, rho, ux, uy, T, n=30):
    x, w = np.polynomial.hermite_e.hermegauss(n)  # weight exp(-x^2/2)
    vx = ux + np.sqrt(T) * x[:, None]
    vy = uy + np.sqrt(T) * x[None, :]
    W = w[:, None] * w[None, :] / (2.0 * np.pi)
    return rho * (W * _row_poly(k, vx, vy)).sum()


def _rows_check(k):
    """The row polynomial itself must be the paper's printed row on the lattice."""
    v = d2v16.velocities().astype(float)
    return np.allclose(_row_poly(k, v[:, 0], v[:, 1]), d2v16.moment_matrix()[k])


@pytest.mark.parametrize("state", STATES)
def test_closed_forms_are_maxwellian_moments(state):
    rho, ux, uy, T = state
    e = rho * (T + 0.5 * (ux * ux + uy * uy))
    fh = eq.feq_hat(np.array(rho), np.array(rho * ux), np.array(rho * uy), np.array(e), 1)
    for k in list(range(11)) + [12, 13]:  # paper k = 1..11, 13, 14
        assert _rows_check(k)
        ref = _maxwellian_moment(k, rho, ux, uy, T)
        scale = max(1.0, abs(ref))
        assert abs(fh[k] - ref) <= 1e-12 * scale * max(1.0, (ux * ux + uy * uy + T) ** 2), (k, fh[k], ref)


@pytest.mark.parametrize("version", [1, 2, 3])
def test_discrete_equilibrium_carries_conserved_moments(version):
    v = d2v16.velocities().astype(float)
    for rho, ux, uy, T in STATES[:4]:
        f = eq.feq(np.array(rho), np.array(ux), np.array(uy), np.array(T), version)
        # explicit velocity sums, not rows of M
        assert np.isclose(f.sum(), rho, rtol=1e-13)
        assert np.isclose((f * v[:, 0]).sum(), rho * ux, rtol=1e-12, atol=1e-12 * rho)
        assert np.isclose((f * v[:, 1]).sum(), rho * uy, rtol=1e-12, atol=1e-12 * rho)
        e = rho * (T + 0.5 * (ux * ux + uy * uy))
        assert np.isclose((f * 0.5 * (v ** 2).sum(1)).sum(), e, rtol=1e-12)


def test_version_rules():
    rho, ux, uy, T = 1.3, 0.4, -0.7, 0.9
    e = rho * (T + 0.5 * (ux * ux + uy * uy))
    args = (np.array(rho), np.array(rho * ux), np.array(rho * uy), np.array(e))
    v1 = eq.feq_hat(*args, version=1)
    v2 = eq.feq_hat(*args, version=2)
    v3 = eq.feq_hat(*args, version=3)
    # version 1: moments 12, 15, 16 vanish; versions differ only there
    assert v1[11] == 0 and v1[14] == 0 and v1[15] == 0
    others = [k for k in range(16) if k not in (11, 14, 15)]
    assert np.array_equal(v1[others], v2[others]) and np.array_equal(v1[others], v3[others])
    assert v2[11] == 0
    # version 3 is M applied to the sampled Maxwellian: at rest it is even in u
    fmax = eq.maxwellian_discrete(rho, 0.0, 0.0, T)
    M = d2v16.moment_matrix()
    assert abs((M[14] * fmax).sum()) < 1e-14 and abs((M[15] * fmax).sum()) < 1e-14


def test_version3_at_rest_is_the_closed_form_of_row_12():
    """At u = 0 the sampled Maxwellian of version 3 is rho/(2 pi T)
    exp(-|v|^2 / 2T) on every velocity of a shell, and row 12 of the printed
    M weighs the shells (|v|^2 = 1, 2, 4, 8) by 1, -4, 16, -64: so
    f^12 = 4 rho / (2 pi T) sum_s w_s exp(-|v_s|^2 / 2T), and rows 15, 16
    (odd in v) vanish."""
    for rho, T in ((1.0, 1.0), (2.5, 0.6), (0.4, 3.0)):
        v3 = eq.feq_hat(np.array(rho), np.array(0.0), np.array(0.0), np.array(rho * T), version=3)
        want = 4.0 * rho / (2.0 * np.pi * T) * sum(w * np.exp(-r2 / (2.0 * T))
                                                   for w, r2 in ((1, 1), (-4, 2), (16, 4), (-64, 8)))
        assert np.isclose(v3[11], want, rtol=1e-13, atol=1e-15)
        assert abs(v3[14]) < 1e-14 and abs(v3[15]) < 1e-14


def test_primitive_inverts_conserved():
    rho, ux, uy, T = 0.7, -1.2, 0.3, 2.5
    e = rho * (T + 0.5 * (ux * ux + uy * uy))
    u1, u2, T1 = eq.primitive(rho, rho * ux, rho * uy, e)
    assert np.allclose([u1, u2, T1], [ux, uy, T], rtol=1e-14)


def _lattice_maps():
    """The square's symmetries acting on the velocities: (matrix g,
    permutation p with v[p[i]] = g v[i])."""
    from oracle import d2v16
    v = d2v16.velocities().astype(int)
    out = []
    for g in (np.array([[0, -1], [1, 0]]), np.array([[1, 0], [0, -1]]), np.array([[0, 1], [1, 0]])):
        p = np.array([int(np.flatnonzero((v == g @ vi).all(axis=1))[0]) for vi in v])
        out.append((g, p))
    return out


@pytest.mark.parametrize("version", [1, 2, 3])
def test_equilibrium_is_covariant_under_the_lattice_symmetries(version):
    """f^eq_i(g u) = f^eq_j(u) with v_i = g v_j, for the 90-degree rotation and
    the reflections of the square lattice (Fig. 1).  The moments of rows 15 and
    16 (v^2 times the third harmonics) must turn into each other under the
    rotation, f^15(R u) = f^16(u) and f^16(R u) = -f^15(u): a sign or a swap
    slipped into one of version 2's two formulas breaks this."""
    rng = np.random.default_rng(31)
    rho = rng.uniform(0.5, 2.0, 50)
    ux, uy = rng.uniform(-0.6, 0.6, (2, 50))
    T = rng.uniform(0.5, 2.0, 50)
    f = eq.feq(rho, ux, uy, T, version)
    for g, p in _lattice_maps():
        gu = g @ np.stack([ux, uy])
        fg = eq.feq(rho, gu[0], gu[1], T, version)
        assert np.allclose(fg[p], f, rtol=1e-13, atol=1e-14)


def test_versions_differ_beyond_navier_stokes_order():
    """Sec. II: the choice of f^12, f^15, f^16 at equilibrium has no effect on
    the macroscopic equations.  The four hydrodynamic eigenvalues of the
    scheme's amplification matrix G(k) (Sec. III) at a moving, non-uniform-rate
    state are the same for versions 1, 2 and 3 up to terms of third order in
    k: their difference falls eightfold per halving of k, while the modes
    themselves move away from 1 at first order."""
    from oracle import fdlb
    from oracle.stability import amplification_matrix
    s = np.array([0, 0, 0, 0, 800, 800, 1200, 1200, 900, 1100, 1000, 950, 1050, 1000, 1000, 1000.0])
    p = fdlb.Params(nx=8, ny=8, dx=1e-2, dy=1e-2, dt=1e-5, s=s)

    def hydro(version, kd):
        p.version = version
        G = amplification_matrix(p, 1.0, 0.3, 0.1, 1.2, kd / p.dx * np.cos(0.3), kd / p.dx * np.sin(0.3))
        ev = np.linalg.eigvals(G)
        ev = ev[np.argsort(np.abs(ev - 1.0))][:4]
        return ev[np.argsort(ev.imag)]

    for other in (2, 3):
        d = [np.abs(hydro(other, kd) - hydro(1, kd)).max() for kd in (0.04, 0.02, 0.01)]
        assert d[0] < 1e-9
        assert 6.0 < d[0] / d[1] < 10.0 and 6.0 < d[1] / d[2] < 10.0, d
    move = [np.abs(hydro(1, kd) - 1.0).max() for kd in (0.02, 0.01)]
    assert 1.8 < move[0] / move[1] < 2.2
