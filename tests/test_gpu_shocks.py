"""The Sod tube (Sec. IV B set-up with the gamma = 2 gas) on the CUDA path
against the exact Riemann solution: small L1 errors at 400 nodes that
shrink under refinement, in FP32 and FP64."""
import numpy as np
import pytest

from oracle import riemann
from paper_1106_0785_gb300 import workloads
from paper_1106_0785_gb300.simulation import Simulation

pytestmark = pytest.mark.gpu

STEPS, DT = 1500, 1e-5  # t = 0.015


def _errors(nx, precision):
    cfg, fields = workloads.sod(nx=nx, ny=4, precision=precision, dt=DT)
    with Simulation(cfg) as sim:
        sim.init_equilibrium(*fields)
        sim.step(STEPS)
        r, u, _, T = sim.macros()
    x = (np.arange(nx) + 0.5) / nx
    re, ue, pe = riemann.exact_riemann((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), (x - 0.5) / (STEPS * DT))
    return np.abs(r[0] - re).mean(), np.abs(u[0] - ue).mean(), np.abs(r[0] * T[0] - pe).mean()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_sod_tube_approaches_the_exact_solution(cuda, precision):
    e400, e800, e1600 = (_errors(n, precision) for n in (400, 800, 1600))
    assert e400[0] < 4e-3 and e400[1] < 1e-2 and e400[2] < 4e-3, e400
    for a, b in ((e400, e800), (e800, e1600)):
        assert all(y < 0.8 * x for x, y in zip(a, b)), (a, b)
