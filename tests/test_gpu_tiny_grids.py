"""Degenerate grids through both step kernels against the FP64 oracle: a
single node, single rows and columns (every neighbour a ghost or the node
itself), grids narrower than one column strip or shorter than one row
segment, and a strip plus one column, for every boundary kind the grid
admits (walls need three nodes across, which the library checks)."""
import numpy as np
import pytest

from oracle import equilibrium as oeq
from oracle import fdlb
from paper_1106_0785_gb300 import mrtlb as M
from paper_1106_0785_gb300.simulation import Simulation
from test_gpu_parity import BCS, KERNELS, _cfg, _input, oracle_params, rel_plane_err

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1), (2, 3), (1, 6), (7, 1), (3, 130), (129, 2)]
SIDES = ["periodic", "outflow_xy", "walls_y", "reflect_y", "diffuse_x", "inflow"]


@pytest.mark.parametrize("kernel", list(KERNELS))
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "%dx%d" % s)
@pytest.mark.parametrize("bc", SIDES)
def test_fp64_tiny_grid_three_steps(cuda, kernel, shape, bc):
    _tiny(kernel, shape, bc, "fp64")


@pytest.mark.parametrize("kernel", list(KERNELS))
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "%dx%d" % s)
@pytest.mark.parametrize("bc", SIDES)
def test_fp32_tiny_grid_three_steps(cuda, kernel, shape, bc):
    """The same in FP32 (the packed-pair march: a pair whose second node is
    outside the grid, strips of one or two columns), from the FP32-rounded
    start, within FP32 rounding of the oracle (2e-6 of the state's scale)."""
    _tiny(kernel, shape, bc, "fp32")


def _tiny(kernel, shape, bc, precision):
    nx, ny = shape
    cfg = _cfg(nx, ny, BCS[bc], precision)
    if bc == "walls_y" and ny < 3:
        with pytest.raises(M.MrtlbError):
            Simulation(cfg)
        return
    (rho, ux, uy, T), nz = _input(cfg, 40)
    p = oracle_params(cfg)
    f0 = fdlb.prepare(oeq.feq(rho, ux, uy, T) + nz, p)
    if precision == "fp32":
        f0 = f0.astype(np.float32).astype(np.float64)
    with Simulation(cfg) as sim:
        sim.set_kernel(KERNELS[kernel])
        sim.set_f(f0.astype(np.float32) if precision == "fp32" else f0)
        sim.step(3)
        g = sim.get_f()
    f = fdlb.run(f0, p, 3)
    assert np.isfinite(g).all()
    if precision == "fp64":
        assert rel_plane_err(g, f) < 1e-11
    else:  # FP32 rounds at the scale of the moments: compare against the state's scale (a single
        # node's fast planes can be 50x smaller than its largest)
        assert np.abs(g - f).max() < 2e-6 * np.abs(f).max()
