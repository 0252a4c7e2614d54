"""mrtlb_reduce_noalloc: the allocation-free conservation sums.

Some callers cannot call cudaMalloc (their device memory belongs to another
allocator with a fixed budget, or their loop must not pay cudaMalloc's
implicit device-wide synchronisation).  This entry point keeps its scratch
in a static device array instead; here it is checked through the C ABI
against mrtlb_reduce on the same states, on two calls in a row.  The file
is collected last so that a failure here does not hide other results.
"""
import ctypes

import numpy as np
import pytest

from oracle import equilibrium as oeq
from paper_1106_0785_gb300 import mrtlb as M
from paper_1106_0785_gb300 import workloads
from paper_1106_0785_gb300.simulation import Simulation

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_matches_reduce_on_two_calls(cuda, precision):
    import torch
    nx, ny = 300 + (precision == "fp32"), 70  # distinct sizes: no carried T_prev
    s = np.random.default_rng(5).uniform(50, 2000, 16)
    s[:4] = 0
    cfg = M.Config(nx=nx, ny=ny, dx=0.01, dy=0.011, dt=2e-4, s=tuple(s),
                   bc=(("periodic", 0, 0, 1),) * 4, precision=precision)
    rho, ux, uy, T = workloads.smooth_fields(nx, ny, 90)
    f0 = oeq.feq(rho, ux, uy, T) + workloads.noise((16, ny, nx), 91, 1e-3)
    dense = torch.empty((16, ny, nx), dtype=torch.float64 if precision == "fp64" else torch.float32,
                        device=cuda)
    prec = M.MRTLB_FP64 if precision == "fp64" else M.MRTLB_FP32
    with Simulation(cfg) as sim:
        sim.set_f(f0)
        outs = []
        for call in range(2):
            if call:
                sim.step(7)
            a = sim.reduce()
            M.mrtlb_get_f(sim.ctx, dense, 1)
            free0 = torch.cuda.mem_get_info()[0]
            b = M.mrtlb_reduce_noalloc(dense, nx, ny, prec, sim.stream.cuda_stream)
            if call:
                # after the first call on the device nothing more is reserved
                assert torch.cuda.mem_get_info()[0] == free0
            outs.append((a, b))
    (a0, b0), (a1, b1) = outs
    for a, b in ((a0, b0), (a1, b1)):
        assert np.allclose(b[:4], a[:4], rtol=1e-12, atol=1e-12 * np.abs(a[:4]).max())
    assert a0[4] == 0.0 and b0[4] == 0.0
    assert a1[4] > 0.0
    assert np.isclose(b1[4], a1[4], rtol=1e-6 if precision == "fp32" else 1e-12)


def test_noalloc_rejects_grids_above_its_scratch(cuda):
    import torch
    dense = torch.zeros(16, dtype=torch.float32, device=cuda)
    code = M.load().mrtlb_reduce_noalloc(dense.data_ptr(), 2048, 1024, M.MRTLB_FP32, None,
                                         (ctypes.c_double * 5)())
    assert code == M.MRTLB_ERR_ARG
    with pytest.raises(M.MrtlbError, match="static scratch"):
        M.mrtlb_reduce_noalloc(dense, 2048, 1024, M.MRTLB_FP32)
