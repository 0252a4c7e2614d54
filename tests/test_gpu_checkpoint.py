"""Checkpoint and resume through the C ABI: a run resumed in a fresh context
from the checkpoint of step n continues bitwise as the uninterrupted run, in
both precisions, on both step kernels and with walls (refilled from the fluid
each step), outflow and inflow sides; corrupted, truncated and mismatched
files are refused and leave the context usable."""
import os

import numpy as np
import pytest

from oracle import equilibrium as oeq
from oracle import fdlb
from paper_1106_0785_gb300 import mrtlb as M
from paper_1106_0785_gb300.simulation import Simulation
from test_gpu_parity import BCS, KERNELS, _cfg, _input, oracle_params

pytestmark = pytest.mark.gpu


def _start(bc, precision):
    cfg = _cfg(150, 37, BCS[bc], precision)
    (rho, ux, uy, T), nz = _input(cfg, 60)
    f0 = fdlb.prepare(oeq.feq(rho, ux, uy, T) + nz, oracle_params(cfg))
    return cfg, (f0 if precision == "fp64" else f0.astype(np.float32))


@pytest.mark.parametrize("kernel", list(KERNELS))
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("bc", ["walls_y", "inflow", "diffuse_x"])
def test_resume_is_bitwise(cuda, tmp_path, kernel, precision, bc):
    cfg, f0 = _start(bc, precision)
    path = str(tmp_path / "state.ck")
    with Simulation(cfg) as sim:
        sim.set_kernel(KERNELS[kernel])
        sim.set_f(f0)
        sim.step(7)
        sim.save(path)
        sim.step(9)
        want = sim.get_f()
    with Simulation(cfg) as sim:
        sim.set_kernel(KERNELS[kernel])
        sim.load(path)
        assert sim.steps == 7
        sim.step(9)
        assert sim.steps == 16
        got = sim.get_f()
    assert np.array_equal(got, want)


def test_bad_checkpoints_are_refused(cuda, tmp_path):
    cfg, f0 = _start("walls_y", "fp32")
    path = str(tmp_path / "state.ck")
    with Simulation(cfg) as sim:
        sim.set_f(f0)
        sim.step(3)
        sim.save(path)
        good = sim.get_f()
    raw = open(path, "rb").read()
    cases = {"corrupt": raw[:200] + bytes([raw[200] ^ 1]) + raw[201:], "truncated": raw[:-9],
             "garbage": b"not a checkpoint" * 4}
    for name, blob in cases.items():
        bad = str(tmp_path / (name + ".ck"))
        open(bad, "wb").write(blob)
        with Simulation(cfg) as sim:
            sim.set_f(f0)
            with pytest.raises(M.MrtlbError):
                sim.load(bad)
            sim.step(3)  # the refused load left the context as it was
            assert np.array_equal(sim.get_f(), good), name
    other = _cfg(150, 37, BCS["walls_y"], "fp32", dt=1e-4)  # another time step
    with Simulation(other) as sim:
        with pytest.raises(M.MrtlbError):
            sim.load(path)
    with Simulation(_cfg(151, 37, BCS["walls_y"], "fp32")) as sim:  # another grid
        with pytest.raises(M.MrtlbError):
            sim.load(path)
    with pytest.raises(M.MrtlbError):
        with Simulation(cfg) as sim:
            sim.load(os.path.join(str(tmp_path), "missing.ck"))
