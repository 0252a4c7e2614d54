"""The Richtmyer-Meshkov trend of Sec. IV B on the CUDA path: with lower
viscosity (larger s5 = s6) or lower heat conductivity (larger s7 = s8) the
shocked interface grows faster.  Measured by the mixing width
W = dx dy sum (rho - its row average)^2 of a 512 x 128 grid (a light/heavy
interface with 8 seeded cosine modes, a Mach-1.5 shock that reaches it at
t = 0.094) at t = 0.3, for viscosity and conductivity each at three levels
(the paper shows the trend, not values; the margins here are 5%)."""
import numpy as np
import pytest

from paper_1106_0785_gb300 import workloads
from paper_1106_0785_gb300.simulation import Simulation

pytestmark = pytest.mark.gpu

NX, NY, DT, K = 512, 128, 1.25e-4, 2400


def _width(s_visc, s_cond):
    amps = list(np.random.default_rng(0).uniform(0.0, 0.02, 8))
    cfg, fields = workloads.richtmyer_meshkov(nx=NX, ny=NY, precision="fp32", dt=DT, x_shock=0.3,
                                              s_visc=s_visc, s_cond=s_cond, s_other=8e3, amplitudes=amps)
    with Simulation(cfg) as sim:
        sim.init_equilibrium(*fields)
        sim.step(K)
        rho = sim.macros()[0]
    dx = 1.0 / NX
    return dx * dx * ((rho - rho.mean(axis=0, keepdims=True)) ** 2).sum()


def test_lower_viscosity_grows_faster(cuda):
    w = [_width(s, 4e3) for s in (2e3, 4e3, 8e3)]  # viscosity rho T / s5: high to low
    assert w[0] * 1.05 < w[1] and w[1] * 1.05 < w[2], w


def test_lower_conductivity_grows_faster(cuda):
    w = [_width(4e3, s) for s in (2e3, 4e3, 8e3)]  # conductivity 2 rho T / s7: high to low
    assert w[0] * 1.05 < w[1] and w[1] * 1.05 < w[2], w
