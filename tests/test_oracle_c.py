"""The oracle's C step (oracle/fdlb_c.c) against the numpy oracle
(oracle/fdlb.py, pinned to the paper in the other oracle tests): the same
method written twice, compared plane by plane after one and after several
steps, for every side the C step implements (periodic, outflow, inflow),
each equilibrium version, and with and without the modification."""
import numpy as np
import pytest

from oracle import cfdlb, fdlb
from oracle import equilibrium as oeq
from paper_1106_0785_gb300 import workloads

SIDES = {
    "periodic": (fdlb.Side(),) * 4,
    "outflow_x": (fdlb.Side(fdlb.OUTFLOW),) * 2 + (fdlb.Side(),) * 2,
    "outflow_xy": (fdlb.Side(fdlb.OUTFLOW),) * 4,
    "inflow_left": (fdlb.Side(fdlb.INFLOW, 0.3, -0.05, 1.2, 1.3), fdlb.Side(fdlb.OUTFLOW)) + (fdlb.Side(),) * 2,
    "inflow_y": (fdlb.Side(),) * 2 + (fdlb.Side(fdlb.INFLOW, 0.02, 0.1, 0.9, 1.1), fdlb.Side(fdlb.OUTFLOW)),
}


def _params(sides, version=1, modified=True, nx=23, ny=17):
    s = np.random.default_rng(3).uniform(100, 3000, 16)
    s[:4] = 0
    return fdlb.Params(nx=nx, ny=ny, dx=0.01, dy=0.012, dt=1e-4, s=s, sides=sides, version=version,
                       modified=modified)


def _state(p, seed):
    rho, ux, uy, T = workloads.smooth_fields(p.nx, p.ny, seed)
    return oeq.feq(rho, ux, uy, T, p.version) + workloads.noise((16, p.ny, p.nx), seed + 1, 1e-3)


def _rel(a, b):
    return (np.abs(a - b).reshape(16, -1).max(1) / np.abs(b).reshape(16, -1).max(1)).max()


@pytest.mark.parametrize("sides", list(SIDES))
@pytest.mark.parametrize("version", [1, 2, 3])
def test_c_step_matches_the_numpy_step(sides, version):
    p = _params(SIDES[sides], version)
    f0 = _state(p, 7)
    assert _rel(cfdlb.step(f0, p), fdlb.step(f0, p)) < 1e-13
    assert _rel(cfdlb.run(f0, p, 6), fdlb.run(f0, p, 6)) < 1e-12


def test_c_step_unmodified_and_ragged_grids():
    for nx, ny in ((1, 1), (2, 5), (40, 3)):
        p = _params(SIDES["inflow_left"], 1, modified=False, nx=nx, ny=ny)
        f0 = _state(p, 11)
        assert _rel(cfdlb.run(f0, p, 3), fdlb.run(f0, p, 3)) < 1e-12


def test_c_step_on_the_bench_crop():
    """The Richtmyer-Meshkov crop the CPU baseline times (inflow left, the
    Mach-1.5 shock and the perturbed interface), 20 steps."""
    cfg, (rho, ux, uy, T) = workloads.richtmyer_meshkov()
    sl = (slice(0, 32), slice(1600, 1728))
    p = fdlb.Params(nx=128, ny=32, dx=cfg.dx, dy=cfg.dy, dt=cfg.dt, s=np.asarray(cfg.s),
                    sides=tuple(fdlb.Side(side[0], *side[1:]) for side in cfg.bc))
    f0 = oeq.feq(rho[sl], ux[sl], uy[sl], T[sl])
    assert _rel(cfdlb.run(f0, p, 20), fdlb.run(f0, p, 20)) < 1e-12


def test_c_step_refuses_sides_it_does_not_implement():
    p = _params((fdlb.Side(fdlb.WALL, 0.1, 0, 1.0),) * 2 + (fdlb.Side(),) * 2)
    assert not cfdlb.supports(p)
    with pytest.raises(ValueError):
        cfdlb.step(np.ones((16, p.ny, p.nx)), p)
