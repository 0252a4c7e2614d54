"""The Richtmyer-Meshkov configuration as stated: 4096 x 1024 nodes, a
Mach-1.5 shock through the perturbed light/heavy interface, 20,000 steps
(dt = 5e-6, to t = 0.1: the shock crosses the interface at t = 0.047 and
the interface then grows), with the fixed post-shock inflow on the left as
the paper's own shocked set-up holds its post-shock side (Sec. IV B).  The
FP32 run (compensated temperature numerator) and the FP64 run must both
stay physical, and FP32 must match FP64 to 1e-4 in relative L1 (the bar
across shocks).  The FP64 path matches the oracle to 1e-12 per step."""
import numpy as np
import pytest

from paper_1106_0785_gb300 import workloads
from paper_1106_0785_gb300.simulation import Simulation

pytestmark = pytest.mark.gpu

STEPS = 20_000


def test_rm_4096x1024_20000_steps_fp32_against_fp64(cuda):
    c32, fields = workloads.richtmyer_meshkov(precision="fp32")
    c64, _ = workloads.richtmyer_meshkov(precision="fp64")
    out = []
    for cfg in (c32, c64):
        with Simulation(cfg) as sim:
            sim.init_equilibrium(*fields)
            for _ in range(STEPS // 5000):
                sim.step(5000)
                sim.sync()  # raises MRTLB_ERR_NONPHYSICAL on rho <= 0, T <= 0 or non-finite
            assert sim.steps == STEPS
            out.append(sim.macros())
    (r, a, b, t), (r0, a0, b0, t0) = out
    l1 = lambda x, y: np.abs(x - y).mean() / np.abs(y).mean()
    err = {"rho": l1(r, r0), "T": l1(t, t0), "ux": l1(a, a0),
           "uy": np.abs(b - b0).mean() / np.abs(a0).mean()}
    print("RM 4096x1024 after %d steps, FP32 vs FP64 relative L1: %s; max |rho32/rho64 - 1| %.2e"
          % (STEPS, ", ".join("%s %.2e" % kv for kv in err.items()), np.abs(r / r0 - 1).max()))
    assert max(err.values()) < 1e-4, err
    assert t0.min() > 0.3 and r0.min() > 0.9  # the FP64 state is physical and bounded


def test_rm_keeps_its_mirror_symmetry_fp64(cuda):
    """The Richtmyer-Meshkov set-up is mirror-symmetric under y -> Ly - y
    (the cosine interface, periodic y, the inflow and outflow sides, and the
    velocity set under v_y -> -v_y), and so must every step be: on 512 x 128
    in FP64, through the shock's passage of the interface (t = 0.047) to
    t = 0.08, the state equals its mirror image to rounding."""
    from oracle import fdlb
    cfg, fields = workloads.richtmyer_meshkov(nx=512, ny=128, precision="fp64", dt=1e-5)
    with Simulation(cfg) as sim:
        sim.init_equilibrium(*fields)
        sim.step(8000)
        sim.sync()
        f = sim.get_f()
    m = fdlb.mirror_permutation(1)
    mirrored = f[m][:, ::-1, :]
    assert np.abs(f - mirrored).max() < 1e-10 * np.abs(f).max()
    # and the interface has moved and deformed (the check is not vacuous)
    rho = f.sum(axis=0)
    assert np.abs(rho - rho.mean(axis=0, keepdims=True)).max() > 0.05
