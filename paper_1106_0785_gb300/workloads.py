"""Seeded synthetic inputs for the paper's three workloads (Sec. IV).

This module builds problem descriptions and initial macroscopic fields only;
it holds none of the lattice Boltzmann arithmetic, so both the CUDA path and
the CPU oracle start from the same numbers and each side forms its own
equilibrium distributions.  Node coordinates are cell centres,
x_i = (i + 1/2) dx, y_j = (j + 1/2) dy, except the Couette channel whose wall
nodes sit on y = 0 and y = 1 (y_j = j dy, dy = 1/(ny - 1)).

Relaxation rates per workload (Pr = s7/s5 = s8/s6):
  Sod        s5..s8 = 1.5e4 (the paper's Riemann viscosity), others 1e5
  Couette    s5 = s6 = 1e2, s7 = s8 = Pr * 1e2, others equal to s5 (as in the
             paper's Couette set-up; with the others ten times s5 the channel
             sheared at U = 0.8 diverges within a few thousand steps for
             every time step tried)
  RM         s5..s8 = 1e4 (the paper's Fig. 7(b) pair), others 1e5;
             dt = 5e-6 on the 4096 x 1024 grid (see richtmyer_meshkov)
  bubble     s5 = s6 in {1e4, 1e3}, s7 = s8 in {1e5, 1e4, 1e3}, others 1e5
             (the six panels of Figs. 7 and 8)
Initial jumps are tanh-smoothed (over 2 cells for Sod and the shock, 3 cells
for the material interface): the central scheme rings a sharp jump into
negative temperatures.
"""
import math

import numpy as np

from .mrtlb import Config

GAMMA = 2.0  # 2D monatomic gas with R = 1: c_v = 1, c_p = 2


def rates(s_visc, s_cond, s_other):
    s = np.full(16, float(s_other))
    s[:4] = 0.0
    s[4] = s[5] = float(s_visc)
    s[6] = s[7] = float(s_cond)
    return tuple(s)


def _smooth_step(x, x0, width):
    return 0.5 * (1.0 + np.tanh((x - x0) / width))


# ---------------------------------------------------------------------------
# Sod shock tube (Sod-type Riemann problem on a thin periodic strip)
# ---------------------------------------------------------------------------
def sod(nx=400, ny=4, precision="fp64", dt=1e-5, left=(1.0, 1.0), right=(0.125, 0.8),
        s_visc=1.5e4, s_cond=1.5e4, s_other=1e5, modified=True):
    """left/right = (rho, T) with u = 0; jump at x = 0.5."""
    dx = 1.0 / nx
    cfg = Config(nx=nx, ny=ny, dx=dx, dy=dx, dt=dt, s=rates(s_visc, s_cond, s_other),
                 bc=(("outflow", 0, 0, 1),) * 2 + (("periodic", 0, 0, 1),) * 2,
                 modified=modified, precision=precision)
    x = (np.arange(nx) + 0.5) * dx
    w = _smooth_step(x, 0.5, 2.0 * dx)
    rho = left[0] + (right[0] - left[0]) * w
    T = left[1] + (right[1] - left[1]) * w
    f = lambda a: np.ascontiguousarray(np.broadcast_to(a[None, :], (ny, nx)))
    zero = np.zeros((ny, nx))
    return cfg, (f(rho), zero.copy(), zero.copy(), f(T))


# ---------------------------------------------------------------------------
# Thermal Couette flow between NEE walls normal to y
# ---------------------------------------------------------------------------
def couette(Pr=1.0, nx=4, ny=200, precision="fp64", dt=1e-4, U=0.8, T0=1.0, T1=1.0,
            s_visc=1e2, s_other=None, modified=True):
    dy = 1.0 / (ny - 1)
    if s_other is None:
        s_other = s_visc
    cfg = Config(nx=nx, ny=ny, dx=dy, dy=dy, dt=dt, s=rates(s_visc, Pr * s_visc, s_other),
                 bc=(("periodic", 0, 0, 1), ("periodic", 0, 0, 1),
                     ("wall", 0.0, 0.0, T0), ("wall", U, 0.0, T1)),
                 modified=modified, precision=precision)
    ones = np.ones((ny, nx))
    T = T0 + (T1 - T0) * (np.arange(ny) * dy)[:, None] * ones
    return cfg, (ones.copy(), np.zeros((ny, nx)), np.zeros((ny, nx)), T)


# ---------------------------------------------------------------------------
# Richtmyer-Meshkov: Mach-1.5 shock onto a perturbed light/heavy interface
# ---------------------------------------------------------------------------
def normal_shock(rho1, p1, mach, g=GAMMA):
    """Post-shock (rho2, u2, p2) and shock speed for a shock moving +x into
    gas at rest: the textbook normal-shock (Rankine-Hugoniot) relations."""
    m2 = mach * mach
    rho2 = rho1 * (g + 1.0) * m2 / ((g - 1.0) * m2 + 2.0)
    p2 = p1 * (2.0 * g * m2 - (g - 1.0)) / (g + 1.0)
    D = mach * math.sqrt(g * p1 / rho1)
    u2 = D * (1.0 - rho1 / rho2)
    return rho2, u2, p2, D


def richtmyer_meshkov(nx=4096, ny=1024, precision="fp32", dt=5e-6, mach=1.5,
                      rho_light=1.0, rho_heavy=3.0, amp=0.02, x_iface=0.5, x_shock=0.4,
                      s_visc=1e4, s_cond=1e4, s_other=1e5, modified=True, amplitudes=None, left="inflow"):
    """Light gas (rho 1) | heavy gas (rho 3), both at p = 1; interface
    x_I(y) = x_iface + sum_k a_k cos(2 pi k y / Ly) (default a_1 = amp).
    Sides: the fixed post-shock state on the left (left="inflow", as the
    paper's own shocked set-up holds its post-shock side) or zero-gradient
    outflow (left="outflow"); outflow on the right; periodic in y.
    dt = 5e-6: at 1e-5 on the 4096 x 1024 grid the FP32 run turns
    non-physical after about 14,700 steps (hot states behind the refracted
    shock are weakly unstable at grid-scale diagonal modes under the
    scheme's amplification matrix, and FP32 rounding seeds them), while
    5e-6 stays physical for 40,000 steps."""
    dx = 1.0 / nx
    Ly = ny * dx
    rho2, u2, p2, _ = normal_shock(rho_light, 1.0, mach)
    if left == "inflow":
        left_side = ("inflow", u2, 0.0, p2 / rho2, rho2)
    elif left == "outflow":
        left_side = ("outflow", 0, 0, 1)
    else:
        raise ValueError("left must be 'inflow' or 'outflow'")
    cfg = Config(nx=nx, ny=ny, dx=dx, dy=dx, dt=dt, s=rates(s_visc, s_cond, s_other),
                 bc=(left_side, ("outflow", 0, 0, 1)) + (("periodic", 0, 0, 1),) * 2,
                 modified=modified, precision=precision)
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dx
    if amplitudes is None:
        amplitudes = [amp]
    xi = np.full(ny, x_iface)
    for k, a in enumerate(amplitudes, start=1):
        xi = xi + a * np.cos(2.0 * math.pi * k * y / Ly)
    w = _smooth_step(x[None, :], xi[:, None], 3.0 * dx)         # 0 light, 1 heavy
    rho = rho_light + (rho_heavy - rho_light) * w
    p = np.ones_like(rho)
    s = 1.0 - _smooth_step(x[None, :], x_shock, 2.0 * dx) * np.ones((ny, 1))  # 1 behind shock
    rho = rho + (rho2 - rho_light) * s
    p = p + (p2 - 1.0) * s
    ux = u2 * s
    T = p / rho
    return cfg, (np.ascontiguousarray(rho), np.ascontiguousarray(ux), np.zeros((ny, nx)),
                 np.ascontiguousarray(T))


# ---------------------------------------------------------------------------
# Random smooth fields for parity tests
# ---------------------------------------------------------------------------
# ---------------------------------------------------------------------------
# Slip Couette flow between diffuse-reflection walls (Sec. IV A, Fig. 3)
# ---------------------------------------------------------------------------
def slip_couette(nx=100, ny=5, precision="fp64", dt=1e-4, d=0.01, U=0.2, Tw=1.0, s_visc=1e2, s_cond=None,
                 s_other=None, version=1):
    """Walls on the x sides (the paper's left and right walls) moving along
    y at -U (left) and +U (right), both at Tw, periodic in y; the fluid
    starts at rest with rho = 1, T = 1.  The paper does not give the rates
    (the slip grows with the Knudsen number); by default all non-conserved
    rates equal s_visc (Pr = 1)."""
    s_cond = s_visc if s_cond is None else s_cond
    s_other = s_visc if s_other is None else s_other
    cfg = Config(nx=nx, ny=ny, dx=d, dy=d, dt=dt, s=rates(s_visc, s_cond, s_other),
                 bc=(("diffuse", 0.0, -U, Tw), ("diffuse", 0.0, U, Tw), ("periodic", 0, 0, 1), ("periodic", 0, 0, 1)),
                 eq_version=version, precision=precision)
    one = np.ones((ny, nx))
    return cfg, (one.copy(), 0 * one, 0 * one, one.copy())


# ---------------------------------------------------------------------------
# Shock-bubble interaction (Sec. IV B, Figs. 7 and 8)
# ---------------------------------------------------------------------------
BUBBLE_PRE = (1.0, 0.0, 0.0, 1.0)            # (rho, u_x, u_y, p) ahead of the shock
BUBBLE_POST = (1.28, -0.3774, 0.0, 1.6512)    # behind the Mach-1.22 shock, moving -x
BUBBLE_GAS = (0.1358, 0.0, 0.0, 1.0)          # the light bubble, in pressure balance


def shock_bubble(nx=600, ny=100, precision="fp32", dt=1e-5, d=0.003, s_visc=1e4, s_cond=1e4,
                 s_other=1e5, radius=25.0, modified=True):
    """A Mach-1.22 shock travelling in -x from the post-shock block
    (node columns 500..nx-1, the paper's 501..600) onto a cylindrical light
    bubble centred at node (449, (ny-1)/2) (the paper's (450, 50), on the
    channel's midline) of `radius` nodes (the paper gives none).  Sides:
    extrapolation (outflow) on the left, the fixed post-shock state on the
    right, reflection on top and bottom.  Interfaces tanh-smoothed over 3
    nodes, the shock over 2."""
    rpost, upost, vpost, ppost = BUBBLE_POST
    cfg = Config(nx=nx, ny=ny, dx=d, dy=d, dt=dt, s=rates(s_visc, s_cond, s_other),
                 bc=(("outflow", 0, 0, 1), ("inflow", upost, vpost, ppost / rpost, rpost),
                     ("reflect", 0, 0, 1), ("reflect", 0, 0, 1)),
                 modified=modified, precision=precision)
    ix = np.arange(nx, dtype=float)[None, :]
    iy = np.arange(ny, dtype=float)[:, None]
    dist = np.sqrt((ix - 449.0) ** 2 + (iy - 0.5 * (ny - 1)) ** 2)
    wb = 1.0 - _smooth_step(dist, radius, 3.0)       # 1 inside the bubble
    ws = _smooth_step(ix + 0.0 * iy, 499.5, 2.0)      # 1 behind the shock
    fields = []
    for k in range(4):
        a = BUBBLE_PRE[k] + (BUBBLE_GAS[k] - BUBBLE_PRE[k]) * wb
        fields.append(a + (BUBBLE_POST[k] - a) * ws)
    rho, ux, uy, p = fields
    return cfg, (rho, ux, uy, p / rho)


def smooth_fields(nx, ny, seed, rho0=1.0, T0=1.0, amp=0.1, umax=0.3, modes=3):
    """Periodic low-mode random fields (rho, ux, uy, T)."""
    rng = np.random.default_rng(seed)
    x = np.arange(nx) / nx
    y = np.arange(ny) / ny

    def field():
        out = np.zeros((ny, nx))
        for _ in range(modes):
            kx, ky = rng.integers(0, 3, size=2)
            ph = rng.uniform(0, 2 * math.pi)
            out += rng.uniform(-1, 1) * np.cos(2 * math.pi * (kx * x[None, :] + ky * y[:, None]) + ph)
        return out / modes

    rho = rho0 * (1.0 + amp * field())
    ux = umax * field()
    uy = umax * field()
    T = T0 * (1.0 + amp * field())
    return rho, ux, uy, T


def noise(shape, seed, scale=1.0):
    """Standard-normal array (e.g. a non-equilibrium perturbation of f)."""
    return scale * np.random.default_rng(seed).standard_normal(shape)


def random_distributions(nx, ny, seed, lo=0.02, hi=0.2):
    """Positive random f of shape (16, ny, nx): a generic input for one step."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(16, ny, nx))


# ---------------------------------------------------------------------------
# Batched set: Sod-type Riemann and Couette instances of uneven shapes
# ---------------------------------------------------------------------------
def batched_instances(n=64, precision="fp32", nx_range=(128, 2048), ny_range=(4, 256)):
    """Instance i draws from numpy.random.default_rng(seed=i): NX ~ U{128..2048},
    NY ~ U{4..256}, Pr ~ U[0.3, 3].  Even i: Sod-type tube, rho 1 | 0.125,
    p 1 | 1/ratio with ratio ~ U[2, 20], dt = 1e-5, s5 = s6 = 1.5e4.  Odd i:
    Couette channel, moving wall speed ~ U[0.1, 0.8], dt = 1e-4, s5 = s6 = 1e2,
    other rates equal to s5.
    s7 = s8 = Pr s5 in both.  Returns a list of (Config, fields)."""
    out = []
    for i in range(n):
        rng = np.random.default_rng(seed=i)
        nx = int(rng.integers(nx_range[0], nx_range[1] + 1))
        ny = int(rng.integers(ny_range[0], ny_range[1] + 1))
        Pr = float(rng.uniform(0.3, 3.0))
        if i % 2 == 0:
            ratio = float(rng.uniform(2.0, 20.0))
            cfg, fields = sod(nx=nx, ny=ny, precision=precision, dt=1e-5, left=(1.0, 1.0),
                              right=(0.125, (1.0 / ratio) / 0.125), s_visc=1.5e4,
                              s_cond=Pr * 1.5e4, s_other=1e5)
        else:
            U = float(rng.uniform(0.1, 0.8))
            cfg, fields = couette(Pr=Pr, nx=nx, ny=ny, precision=precision, dt=1e-4, U=U,
                                  s_visc=1e2)
        out.append((cfg, fields))
    return out
