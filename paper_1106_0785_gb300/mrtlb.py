"""Thin ctypes binding of libmrtlb.so (names follow include/mrtlb.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  PyTorch supplies device memory and streams.  If the library
has not been built, importing the functions raises: there is no fallback.
"""
import ctypes
import os
from dataclasses import dataclass, field

import numpy as np

from . import d2v16

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmrtlb.so")

MRTLB_OK = 0
MRTLB_ERR_ARG = -1
MRTLB_ERR_UNSUPPORTED = -2
MRTLB_ERR_SINGULAR = -3
MRTLB_ERR_CUDA = -4
MRTLB_ERR_NONPHYSICAL = -5
MRTLB_ERR_TIMEOUT = -6
MRTLB_ERR_STATE = -7

MRTLB_BC_PERIODIC = 0
MRTLB_BC_OUTFLOW = 1
MRTLB_BC_WALL_NEE = 2
MRTLB_BC_INFLOW = 3
MRTLB_BC_REFLECT = 4
MRTLB_BC_DIFFUSE = 5

MRTLB_FP32 = 0
MRTLB_FP64 = 1

MRTLB_KERNEL_AUTO = 0
MRTLB_KERNEL_PLAIN = 1
MRTLB_KERNEL_TILED = 2

MRTLB_PEAK_FP32 = 0
MRTLB_PEAK_FP32_PAIR = 1
MRTLB_PEAK_FP64 = 2

# every symbol include/mrtlb.h declares (checked by the CPU test suite)
EXPORTS = (
    "mrtlb_create", "mrtlb_state_bytes", "mrtlb_bind", "mrtlb_init_equilibrium",
    "mrtlb_step", "mrtlb_macros", "mrtlb_reduce", "mrtlb_get_f", "mrtlb_set_f",
    "mrtlb_sync", "mrtlb_set_kernel", "mrtlb_step_count", "mrtlb_last_error",
    "mrtlb_destroy", "mrtlb_timing_begin", "mrtlb_timing_end", "mrtlb_launches_per_step",
    "mrtlb_reduce_noalloc",
    "mrtlb_batch_create", "mrtlb_batch_step", "mrtlb_batch_sync", "mrtlb_batch_set_tiles",
    "mrtlb_batch_get_tiles", "mrtlb_batch_set_graph_steps", "mrtlb_batch_tune", "mrtlb_batch_nodes",
    "mrtlb_batch_last_error", "mrtlb_batch_destroy",
    "mrtlb_set_rates", "mrtlb_get_rates", "mrtlb_selftest_wait", "mrtlb_adjoint_forward", "mrtlb_adjoint_set_interval", "mrtlb_adjoint_backward",
    "mrtlb_adjoint_pass", "mrtlb_adjoint_release", "mrtlb_equilibrium_adjoint", "mrtlb_measure_peak",
    "mrtlb_save", "mrtlb_load",
)

MRTLB_NOALLOC_MAX_NODES = 1 << 20


class MrtlbError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("mrtlb error %d: %s" % (code, msg))
        self.code = code


class mrtlb_bc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("ux", ctypes.c_double),
                ("uy", ctypes.c_double), ("T", ctypes.c_double), ("rho", ctypes.c_double)]


class mrtlb_params(ctypes.Structure):
    _fields_ = [
        ("nvel", ctypes.c_int),
        ("v", ctypes.POINTER(ctypes.c_double)),
        ("M", ctypes.POINTER(ctypes.c_double)),
        ("s", ctypes.POINTER(ctypes.c_double)),
        ("Pr", ctypes.c_double), ("s_visc", ctypes.c_double), ("s_other", ctypes.c_double),
        ("eq_version", ctypes.c_int),
        ("modified", ctypes.c_int),
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dt", ctypes.c_double),
        ("bc", mrtlb_bc * 4),
        ("precision", ctypes.c_int),
        ("stream", ctypes.c_void_p),
    ]


_lib = None


def load(path=LIB_PATH):
    """Load libmrtlb.so; raises if it is missing (build it first)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libmrtlb.so not found at %s: run __graft_entry__.build() "
                           "(the CUDA library is required; there is no CPU path)" % path)
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    lib.mrtlb_create.argtypes = [ctypes.POINTER(mrtlb_params), ctypes.POINTER(P)]
    lib.mrtlb_state_bytes.argtypes = [P, ctypes.POINTER(ctypes.c_size_t)]
    lib.mrtlb_bind.argtypes = [P, P, P, ctypes.c_size_t]
    lib.mrtlb_init_equilibrium.argtypes = [P, P, P, P, P, ctypes.c_int]
    lib.mrtlb_step.argtypes = [P, ctypes.c_long]
    lib.mrtlb_macros.argtypes = [P, P, P, P, P, ctypes.c_int]
    lib.mrtlb_reduce.argtypes = [P, ctypes.POINTER(ctypes.c_double)]
    lib.mrtlb_get_f.argtypes = [P, P, ctypes.c_int]
    lib.mrtlb_set_f.argtypes = [P, P, ctypes.c_int]
    lib.mrtlb_sync.argtypes = [P]
    lib.mrtlb_set_kernel.argtypes = [P, ctypes.c_int]
    lib.mrtlb_step_count.argtypes = [P]
    lib.mrtlb_step_count.restype = ctypes.c_long
    lib.mrtlb_last_error.argtypes = [P]
    lib.mrtlb_last_error.restype = ctypes.c_char_p
    lib.mrtlb_destroy.argtypes = [P]
    lib.mrtlb_destroy.restype = None
    lib.mrtlb_timing_begin.argtypes = [P, ctypes.c_int]
    lib.mrtlb_timing_end.argtypes = [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_long)]
    lib.mrtlb_launches_per_step.argtypes = [P]
    lib.mrtlb_reduce_noalloc.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, P,
                                         ctypes.POINTER(ctypes.c_double)]
    I = ctypes.POINTER(ctypes.c_int)
    lib.mrtlb_batch_create.argtypes = [ctypes.POINTER(P), ctypes.c_int, ctypes.POINTER(P)]
    lib.mrtlb_batch_step.argtypes = [P, ctypes.c_long]
    lib.mrtlb_batch_sync.argtypes = [P]
    lib.mrtlb_batch_set_tiles.argtypes = [P, ctypes.c_int, ctypes.c_int]
    lib.mrtlb_batch_get_tiles.argtypes = [P, I, I, I, I]
    lib.mrtlb_batch_set_graph_steps.argtypes = [P, ctypes.c_int]
    lib.mrtlb_batch_tune.argtypes = [P, ctypes.c_char_p, ctypes.c_int, I, I]
    lib.mrtlb_batch_nodes.argtypes = [P]
    lib.mrtlb_batch_nodes.restype = ctypes.c_longlong
    lib.mrtlb_batch_last_error.argtypes = [P]
    lib.mrtlb_batch_last_error.restype = ctypes.c_char_p
    lib.mrtlb_batch_destroy.argtypes = [P]
    lib.mrtlb_batch_destroy.restype = None
    D = ctypes.POINTER(ctypes.c_double)
    lib.mrtlb_set_rates.argtypes = [P, D]
    lib.mrtlb_get_rates.argtypes = [P, D]
    lib.mrtlb_adjoint_forward.argtypes = [P, ctypes.c_long]
    lib.mrtlb_selftest_wait.argtypes = [P]
    lib.mrtlb_adjoint_set_interval.argtypes = [P, ctypes.c_long]
    lib.mrtlb_adjoint_backward.argtypes = [P, P, P, D, P]
    lib.mrtlb_adjoint_pass.argtypes = [P]
    lib.mrtlb_adjoint_pass.restype = ctypes.c_longlong
    lib.mrtlb_adjoint_release.argtypes = [P]
    lib.mrtlb_equilibrium_adjoint.argtypes = [P] + [P] * 9
    lib.mrtlb_measure_peak.argtypes = [ctypes.c_int, D]
    lib.mrtlb_save.argtypes = [P, ctypes.c_char_p]
    lib.mrtlb_load.argtypes = [P, ctypes.c_char_p]
    _lib = lib
    return lib


def _check(code, ctx=None):
    if code != MRTLB_OK:
        msg = load().mrtlb_last_error(ctx)
        raise MrtlbError(code, msg.decode() if msg else "")


def _ptr(x):
    """Raw pointer of a numpy array, a torch tensor or an int."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


# ----------------------------------------------------------------------------
# Functions with the C names
# ----------------------------------------------------------------------------
def mrtlb_create(params):
    """params: mrtlb_params (see Config.to_params).  Returns an opaque ctx."""
    ctx = ctypes.c_void_p()
    _check(load().mrtlb_create(ctypes.byref(params), ctypes.byref(ctx)))
    return ctx


def mrtlb_state_bytes(ctx):
    n = ctypes.c_size_t()
    _check(load().mrtlb_state_bytes(ctx, ctypes.byref(n)), ctx)
    return n.value


def mrtlb_bind(ctx, f_a, f_b, nbytes):
    _check(load().mrtlb_bind(ctx, _ptr(f_a), _ptr(f_b), nbytes), ctx)


def mrtlb_init_equilibrium(ctx, rho, ux, uy, T, on_device):
    _check(load().mrtlb_init_equilibrium(ctx, _ptr(rho), _ptr(ux), _ptr(uy), _ptr(T),
                                         int(on_device)), ctx)


def mrtlb_step(ctx, nsteps):
    _check(load().mrtlb_step(ctx, int(nsteps)), ctx)


def mrtlb_macros(ctx, rho, ux, uy, T, on_device):
    _check(load().mrtlb_macros(ctx, _ptr(rho), _ptr(ux), _ptr(uy), _ptr(T), int(on_device)), ctx)


def mrtlb_reduce(ctx):
    out = (ctypes.c_double * 5)()
    _check(load().mrtlb_reduce(ctx, out), ctx)
    return np.array(out[:], dtype=np.float64)


def mrtlb_get_f(ctx, f, on_device):
    _check(load().mrtlb_get_f(ctx, _ptr(f), int(on_device)), ctx)


def mrtlb_set_f(ctx, f, on_device):
    _check(load().mrtlb_set_f(ctx, _ptr(f), int(on_device)), ctx)


def mrtlb_sync(ctx):
    _check(load().mrtlb_sync(ctx), ctx)


def mrtlb_selftest_wait(ctx):
    """Returns the status code (MRTLB_ERR_TIMEOUT when the wait bound works)."""
    return load().mrtlb_selftest_wait(ctx)


def mrtlb_set_kernel(ctx, which):
    _check(load().mrtlb_set_kernel(ctx, int(which)), ctx)


def mrtlb_step_count(ctx):
    return load().mrtlb_step_count(ctx)


def mrtlb_last_error(ctx=None):
    return load().mrtlb_last_error(ctx).decode()


def mrtlb_destroy(ctx):
    load().mrtlb_destroy(ctx)


def mrtlb_timing_begin(ctx, max_launches):
    _check(load().mrtlb_timing_begin(ctx, int(max_launches)), ctx)


def mrtlb_timing_end(ctx):
    """(summed step-kernel milliseconds, number of timed launches)"""
    ms = ctypes.c_double()
    n = ctypes.c_long()
    _check(load().mrtlb_timing_end(ctx, ctypes.byref(ms), ctypes.byref(n)), ctx)
    return ms.value, n.value


def mrtlb_save(ctx, path):
    """Write the context's state to a checkpoint file (synchronises)."""
    _check(load().mrtlb_save(ctx, os.fsencode(path)), ctx)


def mrtlb_load(ctx, path):
    """Resume the context from a checkpoint written with the same parameters."""
    _check(load().mrtlb_load(ctx, os.fsencode(path)), ctx)


def mrtlb_measure_peak(kind):
    """Measured fused multiply-add ceiling of the current device in TFLOP/s
    (MRTLB_PEAK_FP32, MRTLB_PEAK_FP32_PAIR or MRTLB_PEAK_FP64)."""
    t = ctypes.c_double()
    rc = load().mrtlb_measure_peak(int(kind), ctypes.byref(t))
    if rc != MRTLB_OK:
        raise MrtlbError(rc, "mrtlb_measure_peak(%d)" % kind)
    return t.value


def mrtlb_reduce_noalloc(f, nx, ny, precision, stream=None):
    """Allocation-free conservation sums of a dense device state
    [16][ny][nx] (see include/mrtlb.h); returns out[0..4]."""
    if nx * ny > MRTLB_NOALLOC_MAX_NODES:
        raise MrtlbError(MRTLB_ERR_ARG, "mrtlb_reduce_noalloc: %d x %d = %d nodes exceeds its static "
                         "scratch of %d nodes" % (nx, ny, nx * ny, MRTLB_NOALLOC_MAX_NODES))
    out = (ctypes.c_double * 5)()
    code = load().mrtlb_reduce_noalloc(_ptr(f), int(nx), int(ny), int(precision), stream, out)
    if code != MRTLB_OK:
        raise MrtlbError(code, "mrtlb_reduce_noalloc failed (%s)" % (
            "bad argument or size above the static scratch limit" if code == MRTLB_ERR_ARG
            else "CUDA error"))
    return np.array(out[:], dtype=np.float64)


def _bcheck(code, b):
    if code != MRTLB_OK:
        msg = load().mrtlb_batch_last_error(b) if b else b""
        raise MrtlbError(code, (msg.decode() if msg else "") or "batch call failed")


def mrtlb_batch_create(ctxs):
    arr = (ctypes.c_void_p * len(ctxs))(*[c.value for c in ctxs])
    b = ctypes.c_void_p()
    code = load().mrtlb_batch_create(arr, len(ctxs), ctypes.byref(b))
    if code != MRTLB_OK:
        raise MrtlbError(code, {MRTLB_ERR_STATE: "every instance must be bound with TMA maps",
                                MRTLB_ERR_ARG: "instances must share precision, stream and parity"}
                         .get(code, "mrtlb_batch_create failed"))
    return b


def mrtlb_batch_step(b, nsteps):
    _bcheck(load().mrtlb_batch_step(b, int(nsteps)), b)


def mrtlb_batch_sync(b):
    _bcheck(load().mrtlb_batch_sync(b), b)


def mrtlb_batch_set_tiles(b, bx, seglen):
    _bcheck(load().mrtlb_batch_set_tiles(b, int(bx), int(seglen)), b)


def mrtlb_batch_get_tiles(b):
    v = [ctypes.c_int() for _ in range(4)]
    _bcheck(load().mrtlb_batch_get_tiles(b, *[ctypes.byref(x) for x in v]), b)
    return tuple(x.value for x in v)  # (bx, seglen, ntiles, grid)


def mrtlb_batch_set_graph_steps(b, steps):
    _bcheck(load().mrtlb_batch_set_graph_steps(b, int(steps)), b)


def mrtlb_batch_tune(b, cache_path=None, trial_steps=8):
    bx = ctypes.c_int()
    sl = ctypes.c_int()
    path = cache_path.encode() if cache_path else None
    _bcheck(load().mrtlb_batch_tune(b, path, int(trial_steps), ctypes.byref(bx), ctypes.byref(sl)), b)
    return bx.value, sl.value


def mrtlb_batch_nodes(b):
    return load().mrtlb_batch_nodes(b)


def mrtlb_batch_last_error(b):
    return load().mrtlb_batch_last_error(b).decode()


def mrtlb_batch_destroy(b):
    load().mrtlb_batch_destroy(b)


def mrtlb_set_rates(ctx, s):
    a = np.ascontiguousarray(np.asarray(s, dtype=np.float64))
    assert a.shape == (16,)
    _check(load().mrtlb_set_rates(ctx, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), ctx)


def mrtlb_get_rates(ctx):
    a = np.zeros(16)
    _check(load().mrtlb_get_rates(ctx, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), ctx)
    return a


def mrtlb_adjoint_forward(ctx, K):
    _check(load().mrtlb_adjoint_forward(ctx, int(K)), ctx)


def mrtlb_adjoint_set_interval(ctx, S):
    _check(load().mrtlb_adjoint_set_interval(ctx, int(S)), ctx)


def mrtlb_adjoint_backward(ctx, dL_dmacros=None, dL_dfK=None, dL_df0=None, want_ds=True):
    """Device FP64 seeds in, (dL/ds numpy[16], or None without want_ds) out;
    dL_df0 (device FP64) filled if given.  Without want_ds the adjoint steps
    skip the rate gradients' work."""
    ds = np.zeros(16) if want_ds else None
    _check(load().mrtlb_adjoint_backward(ctx, _ptr(dL_dmacros), _ptr(dL_dfK),
                                         ds.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if want_ds else None,
                                         _ptr(dL_df0)), ctx)
    return ds


def mrtlb_adjoint_pass(ctx):
    """Id of the forward pass a backward pass would differentiate now (0: none)."""
    return int(load().mrtlb_adjoint_pass(ctx))


def mrtlb_adjoint_release(ctx):
    _check(load().mrtlb_adjoint_release(ctx), ctx)


def mrtlb_equilibrium_adjoint(ctx, dL_df, rho, ux, uy, T, out_rho, out_ux, out_uy, out_T):
    _check(load().mrtlb_equilibrium_adjoint(ctx, *[_ptr(a) for a in (dL_df, rho, ux, uy, T, out_rho, out_ux,
                                                                      out_uy, out_T)]), ctx)


def mrtlb_launches_per_step(ctx):
    n = load().mrtlb_launches_per_step(ctx)
    if n < 0:
        _check(n, ctx)
    return n


# ----------------------------------------------------------------------------
# Parameter marshalling
# ----------------------------------------------------------------------------
BC_NAMES = {"periodic": MRTLB_BC_PERIODIC, "outflow": MRTLB_BC_OUTFLOW, "wall": MRTLB_BC_WALL_NEE,
            "inflow": MRTLB_BC_INFLOW, "reflect": MRTLB_BC_REFLECT, "diffuse": MRTLB_BC_DIFFUSE}


@dataclass
class Config:
    """Problem description handed to mrtlb_create (Sec. II-IV quantities)."""
    nx: int
    ny: int
    dx: float
    dy: float
    dt: float
    s: tuple = None              # 16 rates, or None -> Pr / s_visc / s_other
    Pr: float = 1.0
    s_visc: float = 0.0
    s_other: float = 0.0
    # sides -x, +x, -y, +y: (kind, ux, uy, T) or, for inflow, (kind, ux, uy, T, rho)
    bc: tuple = field(default_factory=lambda: (("periodic", 0, 0, 1),) * 4)
    eq_version: int = 1
    modified: bool = True
    precision: str = "fp32"

    def to_params(self, stream=None):
        p = mrtlb_params()
        keep = []
        v = np.ascontiguousarray(d2v16.velocities().ravel())
        M = np.ascontiguousarray(d2v16.moment_matrix().ravel())
        keep += [v, M]
        dp = ctypes.POINTER(ctypes.c_double)
        p.nvel = 16
        p.v = v.ctypes.data_as(dp)
        p.M = M.ctypes.data_as(dp)
        if self.s is not None:
            s = np.ascontiguousarray(np.asarray(self.s, dtype=np.float64))
            assert s.shape == (16,)
            keep.append(s)
            p.s = s.ctypes.data_as(dp)
        else:
            p.s = None
        p.Pr, p.s_visc, p.s_other = self.Pr, self.s_visc, self.s_other
        p.eq_version = self.eq_version
        p.modified = 1 if self.modified else 0
        p.nx, p.ny = self.nx, self.ny
        p.dx, p.dy, p.dt = self.dx, self.dy, self.dt
        for k, side in enumerate(self.bc):
            kind = BC_NAMES[side[0]] if isinstance(side[0], str) else int(side[0])
            rho = float(side[4]) if len(side) > 4 else 1.0
            p.bc[k] = mrtlb_bc(kind, float(side[1]), float(side[2]), float(side[3]), rho)
        p.precision = MRTLB_FP64 if self.precision == "fp64" else MRTLB_FP32
        p.stream = stream
        p._keep = keep  # keep arrays alive while params are in use
        return p
