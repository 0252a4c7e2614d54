"""One time step of the MRT finite-difference lattice Boltzmann model (oracle).

TEST INFRASTRUCTURE ONLY.

The evolution equation is Eq. 3 (Sec. II):

    d f_i/dt + v_ia d f_i/dx_a = -M^-1_il S_lk (f^_k - f^eq_k)

with the modified energy-flux relaxation of Sec. II (the two rules that
follow Eq. 16c) added to rows k = 7 and 8 of the collision.  The paper
states the space-time discretisation only through its amplification matrix
G (Sec. III).  Reading G term by term (reading R1 in the design notes):

    f_i^{n+1} = f_i^n
              - sum_a (v_ia dt / (2 dx_a)) (f_i(x + e_a) - f_i(x - e_a))
              + sum_a (1/2) (v_ia dt / dx_a)^2 (f_i(x + e_a) - 2 f_i + f_i(x - e_a))
              - dt C_i,
    C = M^-1 c,  c_k = s_k (f^_k - f^eq_k)  (+ the modification for k = 7, 8)

i.e. forward Euler in time with a Lax-Wendroff difference along each axis
and no cross-derivative term.  The velocity gradients inside the
modification are second-order central differences of the time-level-n
velocity at the four cross neighbours (reading R2); rho, T, u in it are the
node's own time-n values (reading R3).

Stages follow the order: walls -> ghost layer -> macroscopic recovery ->
velocity gradients -> moments and equilibria -> collision -> advection ->
update -> walls.  Arrays are laid out (q, y, x): f[q, j, i].

Boundaries (one ghost layer, Sec. IV):
  "periodic"  ghost = the opposite edge (Sec. IV A, IV B);
  "outflow"   zero-gradient extrapolation, ghost = the first interior node
              (the "extrapolation technique", Sec. IV B);
  "wall"      non-equilibrium extrapolation (Sec. IV A): the wall node
              holds f^eq(rho_n, u_w, T_w) + (f - f^eq)(n), n the adjacent
              fluid node, rho_w = rho_n (reading R10).  Wall nodes are not
              advanced by the step; they are refilled from the new adjacent
              row after it.
  "inflow"    a fixed state (Sec. IV B, the shock-bubble's post-shock side):
              ghost = f^eq(rho, u, T) of the side's state.
  "reflect"   specular reflection (Sec. IV B, "reflection conditions"):
              ghost = the first interior node with the velocity set mirrored
              across the side (the normal component of every v_i negated).
  "diffuse"   diffuse reflection (Sec. IV A): velocities entering the fluid
              leave the wall with the equilibrium of the wall state,
              ghost_i = rho_w f^eq_i(1, u_w, T_w); the others copy the edge
              node.  rho_w is the density for which the Lax-Wendroff
              update moves no mass across the side, so the scheme keeps
              the total mass exactly (reading R25).
"""
from dataclasses import dataclass, field

import numpy as np

from . import d2v16
from .equilibrium import conserved, feq, feq_hat, primitive

PERIODIC = "periodic"
OUTFLOW = "outflow"
WALL = "wall"
INFLOW = "inflow"
REFLECT = "reflect"
DIFFUSE = "diffuse"


@dataclass
class Side:
    kind: str = PERIODIC
    ux: float = 0.0   # wall (NEE or diffuse) or inflow velocity
    uy: float = 0.0
    T: float = 1.0    # wall or inflow temperature
    rho: float = 1.0  # inflow density


def mirror_permutation(axis):
    """perm[i] = the velocity index of v_i with component `axis` negated."""
    v = d2v16.velocities()
    w = v.copy()
    w[:, axis] = -w[:, axis]
    return np.array([int(np.flatnonzero((v == wi).all(axis=1))[0]) for wi in w])


@dataclass
class Params:
    nx: int
    ny: int
    dx: float
    dy: float
    dt: float
    s: np.ndarray                      # 16 relaxation rates s_1..s_16
    sides: tuple = field(default_factory=lambda: (Side(), Side(), Side(), Side()))
    version: int = 1                   # equilibrium version for k = 12, 15, 16
    modified: bool = True              # the paper's energy-flux modification

    def __post_init__(self):
        self.s = np.asarray(self.s, dtype=float)
        xm, xp, ym, yp = self.sides
        for a, b in ((xm, xp), (ym, yp)):
            if (a.kind == PERIODIC) != (b.kind == PERIODIC):
                raise ValueError("periodic sides must come in pairs")
        if WALL in (xm.kind, xp.kind) and WALL in (ym.kind, yp.kind):
            raise ValueError("walls on one axis only")


def _walls(f, p):
    """Non-equilibrium extrapolation on wall sides (in place on a copy)."""
    f = f.copy()
    xm, xp, ym, yp = p.sides
    # (side, wall index slicer, adjacent index slicer)
    jobs = []
    if xm.kind == WALL:
        jobs.append((xm, (slice(None), slice(None), 0), (slice(None), slice(None), 1)))
    if xp.kind == WALL:
        jobs.append((xp, (slice(None), slice(None), p.nx - 1), (slice(None), slice(None), p.nx - 2)))
    if ym.kind == WALL:
        jobs.append((ym, (slice(None), 0, slice(None)), (slice(None), 1, slice(None))))
    if yp.kind == WALL:
        jobs.append((yp, (slice(None), p.ny - 1, slice(None)), (slice(None), p.ny - 2, slice(None))))
    for side, w, a in jobs:
        fa = f[a]
        rho, jx, jy, e = conserved(fa)
        ux, uy, T = primitive(rho, jx, jy, e)
        f_neq = fa - feq(rho, ux, uy, T, p.version)
        f[w] = feq(rho, side.ux + 0.0 * rho, side.uy + 0.0 * rho,
                   side.T + 0.0 * rho, p.version) + f_neq
    return f


def _lw_weights(p, axis):
    """Per velocity: the Lax-Wendroff weights of the +e_axis and -e_axis
    neighbours in a node's update (the b - a and b + a of the step)."""
    v = d2v16.velocities()[:, axis].astype(float)
    d = p.dx if axis == 0 else p.dy
    a = v * p.dt / (2.0 * d)
    b = 0.5 * (v * p.dt / d) ** 2
    return b - a, b + a


def _diffuse_ghost(edge, side, axis, sign, p):
    """Diffuse-reflection ghost beside the edge layer edge (16, n); sign = -1
    for the low side of the axis (ghost at -e_axis), +1 for the high side."""
    kp, km = _lw_weights(p, axis)
    # a: weight of the ghost in the edge node's update; b: weight of the edge
    # node in the ghost position's update (the mass the edge hands across)
    a, b = (km, kp) if sign < 0 else (kp, km)
    vn = -sign * d2v16.velocities()[:, axis]          # component along the inward normal
    entering = vn > 0
    one = np.ones(edge.shape[1:])
    e = feq(one, side.ux * one, side.uy * one, side.T * one, p.version)
    num = (b[:, None] * edge).sum(0) - (a[~entering, None] * edge[~entering]).sum(0)
    den = (a[entering, None] * e[entering]).sum(0)
    g = edge.copy()
    g[entering] = (num / den)[None, :] * e[entering]
    return g


def _edge_ghost(edge, side, axis, p, sign=-1):
    """Ghost layer beside a non-periodic side from the adjacent edge layer
    edge (16, n): outflow and walls copy it (behind a wall the ghost is never
    read by an advanced node; the copy keeps it finite), reflect mirrors the
    velocity set across the side, inflow holds f^eq of the side's state,
    diffuse re-emits the wall equilibrium."""
    if side.kind == DIFFUSE:
        return _diffuse_ghost(edge, side, axis, sign, p).astype(edge.dtype)
    if side.kind == REFLECT:
        return edge[mirror_permutation(axis)]
    if side.kind == INFLOW:
        one = np.ones(edge.shape[1:])
        return feq(side.rho * one, side.ux * one, side.uy * one, side.T * one, p.version).astype(edge.dtype)
    return edge.copy()


def _ghosts(f, p):
    """f padded with one ghost node on every side: shape (16, ny+2, nx+2)."""
    nq, ny, nx = f.shape
    g = np.zeros((nq, ny + 2, nx + 2), dtype=f.dtype)
    g[:, 1:-1, 1:-1] = f
    xm, xp, ym, yp = p.sides
    # x sides (rows 1..ny)
    if xm.kind == PERIODIC:
        g[:, 1:-1, 0] = f[:, :, nx - 1]
        g[:, 1:-1, nx + 1] = f[:, :, 0]
    else:
        g[:, 1:-1, 0] = _edge_ghost(f[:, :, 0], xm, 0, p, -1)
        g[:, 1:-1, nx + 1] = _edge_ghost(f[:, :, nx - 1], xp, 0, p, +1)
    if ym.kind == PERIODIC:
        g[:, 0, 1:-1] = f[:, ny - 1, :]
        g[:, ny + 1, 1:-1] = f[:, 0, :]
    else:
        g[:, 0, 1:-1] = _edge_ghost(f[:, 0, :], ym, 1, p, -1)
        g[:, ny + 1, 1:-1] = _edge_ghost(f[:, ny - 1, :], yp, 1, p, +1)
    # corners are not part of the cross stencil; keep them finite
    g[:, 0, 0] = g[:, 1, 1]
    g[:, 0, -1] = g[:, 1, -2]
    g[:, -1, 0] = g[:, -2, 1]
    g[:, -1, -1] = g[:, -2, -2]
    return g


def advanced_mask(p):
    """Boolean (ny, nx): nodes the step advances (all but wall nodes)."""
    m = np.ones((p.ny, p.nx), dtype=bool)
    xm, xp, ym, yp = p.sides
    if xm.kind == WALL:
        m[:, 0] = False
    if xp.kind == WALL:
        m[:, -1] = False
    if ym.kind == WALL:
        m[0, :] = False
    if yp.kind == WALL:
        m[-1, :] = False
    return m


def collision(f, rho, jx, jy, e, grad, p, M=None, Minv=None):
    """C = M^-1 c at each node (Eq. 3 with the Sec. II modification).

    f: (16, ...) distributions; rho, jx, jy, e: conserved moments;
    grad = (dux_dx, dux_dy, duy_dx, duy_dy) at the same nodes.
    """
    if M is None:
        M = d2v16.moment_matrix()
    if Minv is None:
        Minv = d2v16.moment_matrix_inverse()
    s = p.s
    fh = np.tensordot(M, f, axes=(1, 0))
    fheq = feq_hat(rho, jx, jy, e, p.version)
    c = np.zeros_like(fh)
    for k in range(4, 16):
        c[k] = s[k] * (fh[k] - fheq[k])
    if p.modified:
        ux, uy, T = primitive(rho, jx, jy, e)
        dux_dx, dux_dy, duy_dx, duy_dy = grad
        rT = rho * T
        shear = dux_dx - duy_dy          # (du_x/dx - du_y/dy)
        strain = duy_dx + dux_dy         # (du_y/dx + du_x/dy)
        s5, s6, s7, s8 = s[4], s[5], s[6], s[7]
        c[6] = c[6] + (s7 / s5 - 1.0) * rT * ux * shear \
                    + (s7 / s6 - 1.0) * rT * uy * strain
        c[7] = c[7] + (s8 / s6 - 1.0) * rT * ux * strain \
                    + (s8 / s5 - 1.0) * rT * uy * shear
    return np.tensordot(Minv, c, axes=(1, 0))


def step(f, p):
    """Advance f (16, ny, nx) by one time step; returns a new array."""
    M = d2v16.moment_matrix()
    Minv = d2v16.moment_matrix_inverse()
    v = d2v16.velocities().astype(float)

    f = _walls(f, p)
    g = _ghosts(f, p)

    # macroscopic recovery on the padded grid (ghosts included)
    rho_g, jx_g, jy_g, e_g = conserved(g, M)
    ux_g, uy_g, _ = primitive(rho_g, jx_g, jy_g, e_g)

    # second-order central differences at the interior nodes
    dux_dx = (ux_g[1:-1, 2:] - ux_g[1:-1, :-2]) / (2.0 * p.dx)
    duy_dx = (uy_g[1:-1, 2:] - uy_g[1:-1, :-2]) / (2.0 * p.dx)
    dux_dy = (ux_g[2:, 1:-1] - ux_g[:-2, 1:-1]) / (2.0 * p.dy)
    duy_dy = (uy_g[2:, 1:-1] - uy_g[:-2, 1:-1]) / (2.0 * p.dy)

    rho, jx, jy, e = (a[1:-1, 1:-1] for a in (rho_g, jx_g, jy_g, e_g))
    C = collision(f, rho, jx, jy, e, (dux_dx, dux_dy, duy_dx, duy_dy), p, M, Minv)

    # Lax-Wendroff advection along x and y
    A = np.zeros_like(f)
    for q in range(16):
        c = g[q, 1:-1, 1:-1]
        for vel, d, plus, minus in (
            (v[q, 0], p.dx, g[q, 1:-1, 2:], g[q, 1:-1, :-2]),
            (v[q, 1], p.dy, g[q, 2:, 1:-1], g[q, :-2, 1:-1]),
        ):
            if vel == 0.0:
                continue
            a = vel * p.dt / (2.0 * d)
            b = 0.5 * (vel * p.dt / d) ** 2
            A[q] += a * (plus - minus) - b * (plus - 2.0 * c + minus)

    f_new = f - A - p.dt * C
    keep = ~advanced_mask(p)
    f_new[:, keep] = f[:, keep]
    return _walls(f_new, p)


def prepare(f, p):
    """Make wall nodes consistent with their neighbours (idempotent)."""
    return _walls(np.asarray(f), p)


def run(f, p, nsteps):
    for _ in range(nsteps):
        f = step(f, p)
    return f


def macros(f):
    """(rho, ux, uy, T) of a state f (16, ...)."""
    rho, jx, jy, e = conserved(f)
    ux, uy, T = primitive(rho, jx, jy, e)
    return rho, ux, uy, T
