"""The step's reciprocal 1/x (physics.cuh `recip`: the hardware approximation
rcp.approx.ftz.f32 refined by one Newton-Raphson step r <- r (2 - x r)) on
the device, against the correctly rounded reciprocal and CUDA's IEEE
division 1.0f / x, over a sweep of x: normal magnitudes from 2^-40 to 2^40,
the neighbours of powers of two, and the density range of the workloads
(0.05 to 20).  It sets 1/rho in every node update and in the adjoint.
Measured bound: within 1 ulp of the correctly rounded value, equal to it
for most x."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def probe(cuda, tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    out = str(tmp_path_factory.mktemp("recip") / "recip_probe.so")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-shared",
                    "-Xcompiler", "-fPIC", "-o", out, os.path.join(HERE, "probes", "recip_probe.cu")],
                   check=True, capture_output=True)
    lib = ctypes.CDLL(out)
    lib.recip_probe.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
    return lib


def _inputs():
    rng = np.random.default_rng(11)
    x = [np.exp2(rng.uniform(-40, 40, 400_000)),
         rng.uniform(0.05, 20.0, 400_000)]
    # powers of two and their neighbours, up to 64 ulp either side
    p2 = np.exp2(np.arange(-40, 41, dtype=np.float64)).astype(np.float32)
    near = p2.view(np.int32)[:, None] + np.arange(-64, 65, dtype=np.int32)[None, :]
    x.append(near.ravel().view(np.float32))
    x = np.concatenate([np.asarray(a, dtype=np.float32) for a in x])
    return x[np.isfinite(x) & (x > 0)]


def _ulps(a, b):
    return np.abs(a.view(np.int32).astype(np.int64) - b.view(np.int32).astype(np.int64))


def test_recip_within_one_ulp_of_the_correctly_rounded_reciprocal(probe):
    x = _inputs()
    n = x.size
    out = np.empty(4 * n, dtype=np.float32)
    assert probe.recip_probe(x.ctypes.data, out.ctypes.data, n) == 0
    scalar, lane_x, lane_y, div = out.reshape(4, n)
    exact = (1.0 / x.astype(np.float64)).astype(np.float32)  # correctly rounded (no ties at these x)
    assert np.array_equal(div, exact)                       # CUDA's IEEE division is correctly rounded
    for r in (scalar, lane_x, lane_y):
        u = _ulps(r, exact)
        assert u.max() <= 1, (u.max(), x[np.argmax(u)])
    assert np.array_equal(lane_x, scalar) and np.array_equal(lane_y, scalar)  # packed lanes round alike
    frac_exact = float((_ulps(scalar, exact) == 0).mean())
    print("recip: max 1 ulp, %.4f of x correctly rounded" % frac_exact)
    assert frac_exact > 0.5
    # the workloads' density range on its own
    m = (x >= 0.05) & (x <= 20.0)
    assert _ulps(scalar[m], exact[m]).max() <= 1
