"""The C ABI without a GPU: the library builds for sm_103a, loads, exports
every entry point include/mrtlb.h declares, and mrtlb_create (host-only)
validates its arguments."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1106_0785_gb300 import d2v16 as pd
from paper_1106_0785_gb300 import mrtlb as M
from paper_1106_0785_gb300 import workloads

HEADER_DIR = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include")


def _declared():
    names = set()
    for fn in os.listdir(HEADER_DIR):
        if fn.endswith(".h"):
            text = open(os.path.join(HEADER_DIR, fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(mrtlb_\w+)\s*\(", text))
    return names


def test_header_declarations_are_exported(lib):
    declared = _declared()
    assert declared, "no declarations found"
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(M.EXPORTS)


def _create(cfg):
    ctx = ctypes.c_void_p()
    p = cfg.to_params()
    rc = M.load().mrtlb_create(ctypes.byref(p), ctypes.byref(ctx))
    return rc, ctx


def test_create_accepts_the_paper_workloads(lib):
    for cfg, _ in (workloads.sod(), workloads.couette(2.0), workloads.richtmyer_meshkov(nx=256, ny=64)):
        rc, ctx = _create(cfg)
        assert rc == M.MRTLB_OK, M.mrtlb_last_error(None)
        nbytes = M.mrtlb_state_bytes(ctx)
        esize = 8 if cfg.precision == "fp64" else 4
        assert nbytes >= 16 * (cfg.ny + 2) * (cfg.nx + 2) * esize
        M.mrtlb_destroy(ctx)


def test_create_rejects_other_velocity_sets_and_matrices(lib):
    cfg, _ = workloads.sod()
    p = cfg.to_params()
    Mbad = pd.moment_matrix().copy()
    Mbad[5, 4] += 1.0
    Mbad = np.ascontiguousarray(Mbad.ravel())
    p.M = Mbad.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    ctx = ctypes.c_void_p()
    assert M.load().mrtlb_create(ctypes.byref(p), ctypes.byref(ctx)) == M.MRTLB_ERR_UNSUPPORTED
    assert not ctx.value
    assert "M[6][5]" in M.mrtlb_last_error(None)
    p = cfg.to_params()
    v = pd.velocities()[[1, 0] + list(range(2, 16))].ravel().copy()
    p.v = v.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert M.load().mrtlb_create(ctypes.byref(p), ctypes.byref(ctx)) == M.MRTLB_ERR_UNSUPPORTED
    p = cfg.to_params()
    p.nvel = 9
    assert M.load().mrtlb_create(ctypes.byref(p), ctypes.byref(ctx)) == M.MRTLB_ERR_UNSUPPORTED


@pytest.mark.parametrize("change,code", [
    (dict(dt=1e-2), M.MRTLB_ERR_ARG),                       # CFL 2 dt / dx > 1
    (dict(s=tuple([0] * 4 + [3e5] * 12)), M.MRTLB_ERR_ARG),  # s dt > 2
    (dict(nx=0), M.MRTLB_ERR_ARG),
    (dict(eq_version=4), M.MRTLB_ERR_ARG),
    (dict(bc=(("periodic", 0, 0, 1), ("outflow", 0, 0, 1)) + (("periodic", 0, 0, 1),) * 2),
     M.MRTLB_ERR_ARG),                                      # unpaired periodic side
    (dict(bc=(("wall", 0, 0, 1),) * 4), M.MRTLB_ERR_UNSUPPORTED),  # walls on both axes
    (dict(s=tuple([0] * 4 + [0.0] * 12)), M.MRTLB_ERR_ARG),  # modified needs s5, s6 > 0
])
def test_create_rejects_bad_arguments(lib, change, code):
    cfg, _ = workloads.sod()
    for k, v in change.items():
        setattr(cfg, k, v)
    rc, ctx = _create(cfg)
    assert rc == code, M.mrtlb_last_error(None)
    assert not ctx.value
    assert M.mrtlb_last_error(None)


def test_rates_derived_from_prandtl(lib):
    cfg, _ = workloads.couette(2.0)
    cfg.s = None
    cfg.Pr, cfg.s_visc, cfg.s_other = 2.0, 100.0, 1000.0
    rc, ctx = _create(cfg)
    assert rc == M.MRTLB_OK
    M.mrtlb_destroy(ctx)


def test_calls_before_bind_are_rejected(lib):
    cfg, _ = workloads.sod()
    rc, ctx = _create(cfg)
    assert rc == M.MRTLB_OK
    assert M.load().mrtlb_step(ctx, 1) == M.MRTLB_ERR_STATE
    assert "bind" in M.mrtlb_last_error(ctx)
    M.mrtlb_destroy(ctx)


def test_binding_fails_loudly_without_the_library(tmp_path):
    saved = M._lib
    try:
        M._lib = None
        with pytest.raises(RuntimeError, match="libmrtlb.so not found"):
            M.load(str(tmp_path / "libmrtlb.so"))
    finally:
        M._lib = saved


def test_header_is_plain_c_and_links(lib, tmp_path):
    """A C99 program (no C++) includes include/mrtlb.h under -pedantic
    -Werror, links against libmrtlb.so and runs the calls that need no GPU:
    argument errors and the error-string call."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    src = tmp_path / "use_header.c"
    src.write_text(r'''
#include "mrtlb.h"
#include <stdio.h>
int main(void) {
  mrtlb_ctx* ctx = NULL;
  double out[5];
  if (mrtlb_create(NULL, &ctx) != MRTLB_ERR_ARG) return 1;
  if (mrtlb_step(NULL, 1) != MRTLB_ERR_ARG) return 2;
  if (mrtlb_reduce(NULL, out) != MRTLB_ERR_ARG) return 3;
  if (mrtlb_adjoint_pass(NULL) != 0) return 4;
  if (mrtlb_last_error(NULL) == NULL) return 5;
  printf("ok\n");
  return 0;
}
''')
    libdir = os.path.dirname(M.LIB_PATH)
    exe = tmp_path / "use_header"
    subprocess.run([cc, "-std=c99", "-pedantic", "-Wall", "-Wextra", "-Werror", "-I", HEADER_DIR, str(src),
                    "-L", libdir, "-lmrtlb", "-Wl,-rpath," + libdir, "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and r.stdout.strip() == "ok", (r.returncode, r.stdout, r.stderr)
