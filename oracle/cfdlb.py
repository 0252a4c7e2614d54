"""The oracle's time step in plain C (fdlb_c.c), for speed on the host.

TEST INFRASTRUCTURE ONLY.

Same method, stage order and arithmetic definitions as fdlb.py (Eq. 3 with
the Sec. II modification, discretised as Sec. III's G reads), written as
plain FP64 loops and compiled with gcc -O3 (no intrinsics, no
machine-specific flags).  It covers the sides the timed Richtmyer-Meshkov
crop uses (periodic, outflow, inflow); fdlb.py remains the reference for
walls and reflecting or diffuse sides.  Pinned against fdlb.py step by step
(tests/test_oracle_c.py).  M and M^-1 come from d2v16 (the exact rationals).
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np

from . import d2v16

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "fdlb_c.c")
LIB = os.path.join(HERE, "_build", "libfdlb_c.so")
KINDS = {"periodic": 0, "outflow": 1, "inflow": 3}

_lib = None


def build(force=False):
    """Compile fdlb_c.c into oracle/_build/libfdlb_c.so (if out of date)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cc = os.environ.get("CC") or shutil.which("gcc") or shutil.which("cc")
    if not cc:
        raise RuntimeError("no C compiler for the oracle's C step")
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    tmp = LIB + ".%d.tmp" % os.getpid()
    subprocess.run([cc, "-O3", "-std=c99", "-fPIC", "-shared", "-o", tmp, SRC, "-lm"], check=True,
                   capture_output=True)
    os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        D = ctypes.POINTER(ctypes.c_double)
        I = ctypes.POINTER(ctypes.c_int)
        lib.oracle_step.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                    D, ctypes.c_int, ctypes.c_int, I, D, D, D, D, D, D]
        lib.oracle_run.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                   D, ctypes.c_int, ctypes.c_int, I, D, D, D, D, ctypes.c_long, D]
        _lib = lib
    return _lib


def supports(p):
    """True when every side of fdlb.Params p is one the C step implements."""
    return all(side.kind in KINDS for side in p.sides)


class _Args:
    def __init__(self, p, shape):
        if not supports(p):
            raise ValueError("the C step implements periodic, outflow and inflow sides only")
        nq, ny, nx = shape
        if (nq, ny, nx) != (16, p.ny, p.nx):
            raise ValueError("f must be (16, ny, nx)")
        D = ctypes.POINTER(ctypes.c_double)
        self.s = np.ascontiguousarray(p.s, dtype=np.float64)
        self.kinds = np.array([KINDS[side.kind] for side in p.sides], dtype=np.int32)
        self.side = np.array([[side.ux, side.uy, side.T, side.rho] for side in p.sides], dtype=np.float64)
        self.M = np.ascontiguousarray(d2v16.moment_matrix())
        self.Minv = np.ascontiguousarray(d2v16.moment_matrix_inverse())
        npad = (nx + 2) * (ny + 2)
        self.work = np.empty(16 * nx * ny + 19 * npad + 4 * nx * ny, dtype=np.float64)
        self.head = (nx, ny, p.dx, p.dy, p.dt, self.s.ctypes.data_as(D), int(p.version), int(bool(p.modified)),
                     self.kinds.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), self.side.ctypes.data_as(D),
                     self.M.ctypes.data_as(D), self.Minv.ctypes.data_as(D))


class Runner:
    """Steps one problem in place, reusing its work arrays between calls."""

    def __init__(self, f, p):
        self.a = _Args(p, f.shape)
        self.f = np.array(f, dtype=np.float64, order="C", copy=True)

    def run(self, nsteps):
        D = ctypes.POINTER(ctypes.c_double)
        rc = _load().oracle_run(*self.a.head, self.f.ctypes.data_as(D), int(nsteps), self.a.work.ctypes.data_as(D))
        if rc:
            raise RuntimeError("oracle_run failed (%d)" % rc)
        return self.f


def run(f, p, nsteps):
    """nsteps steps of fdlb.Params p from f (16, ny, nx); returns a new array."""
    return Runner(f, p).run(nsteps).copy()


def step(f, p):
    """One step; returns a new array."""
    return run(f, p, 1)
