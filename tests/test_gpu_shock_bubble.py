"""The paper's shock-bubble set-up (Sec. IV B) on the CUDA path: inflow,
outflow and reflecting sides together, against the oracle, the set-up's
mirror symmetry, and a run that carries the shock through the bubble."""
import numpy as np
import pytest

from oracle import equilibrium as oeq
from oracle import fdlb
from paper_1106_0785_gb300 import workloads
from paper_1106_0785_gb300.simulation import Simulation

pytestmark = pytest.mark.gpu

KINDS = {"outflow": fdlb.OUTFLOW, "inflow": fdlb.INFLOW, "reflect": fdlb.REFLECT}


def _oracle_params(cfg):
    sides = tuple(fdlb.Side(KINDS[side[0]], *side[1:]) for side in cfg.bc)
    return fdlb.Params(nx=cfg.nx, ny=cfg.ny, dx=cfg.dx, dy=cfg.dy, dt=cfg.dt, s=np.asarray(cfg.s),
                       sides=sides, modified=cfg.modified)


def test_shock_bubble_fp32_matches_oracle(cuda):
    cfg, (rho, ux, uy, T) = workloads.shock_bubble(precision="fp32")
    with Simulation(cfg) as sim:
        sim.init_equilibrium(rho, ux, uy, T)
        sim.step(300)
        r, a, b, t = sim.macros()
    ro, ao, bo, to = fdlb.macros(fdlb.run(oeq.feq(rho, ux, uy, T), _oracle_params(cfg), 300))
    l1 = lambda x, y: np.abs(x - y).mean() / np.abs(y).mean()
    assert l1(r, ro) < 1e-5 and l1(t, to) < 1e-5, (l1(r, ro), l1(t, to))
    # velocity across the shock front: L1, as for the other shocked runs
    assert np.abs(a - ao).mean() < 1e-4 * np.abs(ao).mean(), np.abs(a - ao).mean() / np.abs(ao).mean()


def test_shock_bubble_keeps_its_mirror_symmetry_fp64(cuda):
    """Symmetric about the channel's midline at any time: the reflecting
    sides and the step commute with the mirror.  6000 steps take the shock
    into the bubble."""
    cfg, fields = workloads.shock_bubble(precision="fp64")
    with Simulation(cfg) as sim:
        sim.init_equilibrium(*fields)
        sim.step(6000)
        f = sim.get_f()
    m = fdlb.mirror_permutation(1)
    mirrored = f[m][:, ::-1, :]
    assert np.abs(f - mirrored).max() < 1e-10 * np.abs(f).max()


def test_shock_passes_the_bubble_fp32(cuda):
    """30,000 steps (t = 0.3): the state stays physical, the shock has
    compressed the gas beyond the post-shock density, and the bubble has
    been carried downstream (in -x) by the post-shock flow."""
    cfg, fields = workloads.shock_bubble(precision="fp32")
    light = lambda r: (r < 0.6)
    ix = np.arange(cfg.nx)[None, :]
    with Simulation(cfg) as sim:
        sim.init_equilibrium(*fields)
        r0 = sim.macros()[0]
        sim.step(30000)
        sim.sync()  # raises on a non-physical state
        r, a, b, t = sim.macros()
    assert np.isfinite(r).all() and r.min() > 0 and t.min() > 0
    assert r.max() > 1.3
    x0 = (ix * light(r0)).sum() / light(r0).sum()
    x1 = (ix * light(r)).sum() / light(r).sum()
    assert x1 < x0 - 10, (x0, x1)
