"""The seeded input generators: shapes, physical ranges, and the RM
post-shock state against the oracle's own jump-condition solver."""
import numpy as np

from oracle import riemann
from paper_1106_0785_gb300 import workloads


def test_normal_shock_relations_agree_with_jump_condition_solver():
    for mach in (1.22, 1.5, 3.0):
        a = workloads.normal_shock(1.0, 1.0, mach)
        b = riemann.shock_state(1.0, 1.0, mach)
        assert np.allclose(a, b, rtol=1e-10)


def test_richtmyer_meshkov_inputs():
    cfg, (rho, ux, uy, T) = workloads.richtmyer_meshkov(nx=512, ny=128)
    assert rho.shape == (128, 512)
    p = rho * T
    # light gas at rest at p = 1 ahead of the shock, heavy gas (rho 3) beyond the interface
    x = (np.arange(512) + 0.5) / 512
    assert np.allclose(p[:, (x > 0.45) & (x < 0.46)], 1.0, atol=1e-6)
    assert np.allclose(rho[:, x > 0.6], 3.0, atol=1e-6)
    # post-shock state behind x = 0.4
    r2, u2, p2, _ = workloads.normal_shock(1.0, 1.0, 1.5)
    assert np.allclose(rho[:, x < 0.35], r2) and np.allclose(ux[:, x < 0.35], u2)
    assert np.allclose(p[:, x < 0.35], p2)
    assert (uy == 0).all() and (T > 0).all()
    # the interface is displaced by the cosine (two rows differ)
    assert not np.allclose(rho[0], rho[64])
    assert 2 * cfg.dt / cfg.dx <= 1.0


def test_sod_and_couette_inputs():
    cfg, (rho, ux, uy, T) = workloads.sod()
    assert rho.shape == (4, 400) and rho[0, 0] > 0.99 and rho[0, -1] < 0.126
    assert np.allclose(rho[0], rho[3])
    cfg, (rho, ux, uy, T) = workloads.couette(0.5)
    assert rho.shape == (200, 4) and (rho == 1).all() and (T == 1).all()
    assert cfg.s[6] == 0.5 * cfg.s[4]
    assert cfg.bc[3][1] == 0.8


def test_generators_are_seeded():
    a = workloads.smooth_fields(40, 30, seed=3)
    b = workloads.smooth_fields(40, 30, seed=3)
    c = workloads.smooth_fields(40, 30, seed=4)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    assert not np.array_equal(a[0], c[0])
    assert (a[0] > 0).all() and (a[3] > 0).all()
