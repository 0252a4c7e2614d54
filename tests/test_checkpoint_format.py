"""The checkpoint file without a GPU: files written here from the layout
include/mrtlb.h and csrc/checkpoint.cu document (magic, version, precision,
grid, step count, a 64-bit FNV-1a hash of the step's parameters, the dense
state, an FNV-1a checksum) pass mrtlb_load's validation when they are
right, and each wrong field is refused with its own reason.  A context that
was created but not bound reaches the state copy only after validation, so
MRTLB_ERR_STATE there means the file was accepted."""
import ctypes
import struct

import numpy as np
import pytest

from paper_1106_0785_gb300 import mrtlb as M
from paper_1106_0785_gb300 import workloads

FNV_OFFSET, FNV_PRIME = 14695981039346656037, 1099511628211
KINDS = {"periodic": 0, "outflow": 1, "wall": 2, "inflow": 3, "reflect": 4, "diffuse": 5}


def fnv1a(data, h=FNV_OFFSET):
    for b in data:
        h = ((h ^ b) * FNV_PRIME) & 0xFFFFFFFFFFFFFFFF
    return h


def params_hash(cfg, rates):
    b = struct.pack("<3i", cfg.nx, cfg.ny, 1 if cfg.precision == "fp64" else 0)
    b += struct.pack("<3d", cfg.dx, cfg.dy, cfg.dt)
    b += struct.pack("<16d", *rates)
    b += struct.pack("<2i", cfg.eq_version, 1 if cfg.modified else 0)
    for side in cfg.bc:
        kind, ux, uy, T = side[:4]
        rho = side[4] if len(side) > 4 else 1.0
        b += struct.pack("<i4d", KINDS[kind], ux, uy, T, rho)
    return fnv1a(b)


def checkpoint_bytes(cfg, rates, steps=5, data=None, **over):
    es = 8 if cfg.precision == "fp64" else 4
    nbytes = 16 * cfg.nx * cfg.ny * es
    if data is None:
        data = np.random.default_rng(1).uniform(0.01, 0.1, nbytes // es).astype("<f8" if es == 8 else "<f4").tobytes()
    f = dict(magic=b"MRTLBCK1", version=1, prec=1 if es == 8 else 0, nx=cfg.nx, ny=cfg.ny, steps=steps,
             hash=params_hash(cfg, rates), nbytes=nbytes, checksum=fnv1a(data))
    f.update(over)
    head = f["magic"] + struct.pack("<4Iq2Q", f["version"], f["prec"], f["nx"], f["ny"], f["steps"], f["hash"],
                                    f["nbytes"])
    return head + data + struct.pack("<Q", f["checksum"])


@pytest.fixture
def ctx(lib):
    cfg, _ = workloads.couette(Pr=2.0, nx=6, ny=9, precision="fp32")
    c = ctypes.c_void_p()
    p = cfg.to_params()
    assert lib.mrtlb_create(ctypes.byref(p), ctypes.byref(c)) == M.MRTLB_OK, M.mrtlb_last_error(None)
    yield cfg, c, M.mrtlb_get_rates(c)
    M.mrtlb_destroy(c)


def _load(lib, c, path):
    return lib.mrtlb_load(c, str(path).encode())


def test_a_right_file_passes_validation(lib, ctx, tmp_path):
    cfg, c, rates = ctx
    path = tmp_path / "ok.ck"
    path.write_bytes(checkpoint_bytes(cfg, rates))
    assert _load(lib, c, path) == M.MRTLB_ERR_STATE  # validated, then refused: not bound
    assert "bind" in M.mrtlb_last_error(c)


@pytest.mark.parametrize("change,reason", [
    (dict(magic=b"MRTLBCK0"), "not a checkpoint"),
    (dict(version=2), "version"),
    (dict(prec=1), "another grid or precision"),
    (dict(nx=7), "another grid or precision"),
    (dict(hash=123), "other parameters"),
    (dict(nbytes=8), "size mismatch"),
    (dict(checksum=1), "checksum mismatch"),
])
def test_each_wrong_field_is_refused(lib, ctx, tmp_path, change, reason):
    cfg, c, rates = ctx
    path = tmp_path / "bad.ck"
    path.write_bytes(checkpoint_bytes(cfg, rates, **change))
    assert _load(lib, c, path) == M.MRTLB_ERR_ARG
    assert reason in M.mrtlb_last_error(c)


def test_other_rates_change_the_hash(lib, ctx, tmp_path):
    cfg, c, rates = ctx
    other = rates.copy()
    other[6] *= 1.5
    path = tmp_path / "rates.ck"
    path.write_bytes(checkpoint_bytes(cfg, other))
    assert _load(lib, c, path) == M.MRTLB_ERR_ARG
    assert "other parameters" in M.mrtlb_last_error(c)


def test_truncated_and_missing_files(lib, ctx, tmp_path):
    cfg, c, rates = ctx
    path = tmp_path / "short.ck"
    path.write_bytes(checkpoint_bytes(cfg, rates)[:-3])
    assert _load(lib, c, path) == M.MRTLB_ERR_ARG and "truncated" in M.mrtlb_last_error(c)
    assert _load(lib, c, tmp_path / "missing.ck") == M.MRTLB_ERR_ARG
    assert lib.mrtlb_save(c, str(tmp_path / "x.ck").encode()) == M.MRTLB_ERR_STATE  # nothing bound
