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


def test_plane_offsets_beyond_32_bits(cuda):
    """A grid whose distribution offsets pass 2^31 elements (12288 x 12000
    nodes: planes of 1.48e8 padded nodes, so plane 15 starts past 2.2e9;
    9.4 GB per FP32 state): the equilibrium set on the device, one step of
    the FP32 march, and the nodes nearest the end of the grid plus random
    ones checked against the oracle's step of their 3 x 3 neighbourhood
    (the same equilibrium in FP64)."""
    from paper_1106_0785_gb300 import workloads
    nx, ny = 12288, 12000
    cfg, (rho, ux, uy, T) = workloads.richtmyer_meshkov(nx=nx, ny=ny, precision="fp32", dt=5e-6 * 4096 / nx)
    with Simulation(cfg) as sim:
        assert sim.state_bytes >= 16 * (ny + 2) * (nx + 2) * 4 and (ny + 2) * (nx + 2) * 15 > 2 ** 31
        sim.set_kernel(M.MRTLB_KERNEL_TILED)
        sim.init_equilibrium(rho, ux, uy, T)
        sim.step(1)
        out = sim.get_f()
    rng = np.random.default_rng(9)
    xs = list(rng.integers(1, nx - 1, 400)) + [nx - 2, nx - 2, nx - 130, 1, 127, 128]
    ys = list(rng.integers(1, ny - 1, 400)) + [ny - 2, ny - 3, ny - 2, ny - 2, 6000, 11999 - 1]
    K = len(xs)
    patch = lambda a: np.concatenate([a[y - 1:y + 2, x - 1:x + 2] for x, y in zip(xs, ys)], axis=1)
    f = oeq.feq(patch(rho), patch(ux), patch(uy), patch(T))  # (16, 3, 3K)
    p = oracle_params(cfg)
    pp = fdlb.Params(nx=3 * K, ny=3, dx=p.dx, dy=p.dy, dt=p.dt, s=p.s, modified=p.modified)
    ref = fdlb.step(f, pp)[:, 1, 1::3]
    got = out[:, ys, xs].astype(np.float64)
    scale = np.abs(ref).max(axis=1, keepdims=True)
    assert (np.abs(got - ref) / scale).max() < 2e-6
