"""The tallest grid the library accepts (65535 rows, the limit of the CUDA
grid dimension the row segments use) through both step kernels, one step
against the FP64 oracle over the whole grid, in both precisions."""
import numpy as np
import pytest

from oracle import equilibrium as oeq
from oracle import fdlb
from paper_1106_0785_gb300 import mrtlb as M
from paper_1106_0785_gb300.simulation import Simulation
from test_gpu_parity import BCS, KERNELS, _cfg, _input, oracle_params, rel_plane_err

pytestmark = pytest.mark.gpu

NX, NY = 24, 65535


@pytest.fixture(scope="module")
def case():
    cfg = _cfg(NX, NY, BCS["outflow_x"], "fp64")
    (rho, ux, uy, T), nz = _input(cfg, 50)
    p = oracle_params(cfg)
    f0 = fdlb.prepare(oeq.feq(rho, ux, uy, T) + nz, p)
    return cfg, f0, fdlb.step(f0, p)


@pytest.mark.parametrize("kernel", list(KERNELS))
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-6)])
def test_one_step_on_the_tallest_grid(cuda, case, kernel, precision, tol):
    cfg, f0, f1 = case
    cfg.precision = precision
    with Simulation(cfg) as sim:
        sim.set_kernel(KERNELS[kernel])
        sim.set_f(f0 if precision == "fp64" else f0.astype(np.float32))
        sim.step(1)
        g = sim.get_f().astype(np.float64)
    assert rel_plane_err(g, f1) < tol


def test_one_row_more_is_rejected(cuda):
    with pytest.raises(M.MrtlbError):
        Simulation(_cfg(NX, NY + 1, BCS["outflow_x"], "fp32"))
