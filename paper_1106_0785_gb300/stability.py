"""Linear stability of the implemented step (Sec. III) from the library itself.

For a uniform state (rho, u, T) the step is translation invariant, so its
linearisation maps a Fourier mode exp(i k x) w to exp(i k x) G(k) w with
the amplification matrix G of Sec. III.  This module measures G on the GPU
through the library's own FP64 step: the uniform state is perturbed at one
node along velocity q (central differences, +-eps), stepped once, and the
response's discrete Fourier transform along the axis is column q of G(k)
for every k = 2 pi m / (n d), m = 0..n/2, at once.  Sixteen pairs of one-step
runs on an n-node periodic strip give the whole spectrum.  The scheme is
linearly stable for the state when max_k max |eig G(k)| <= 1.
"""
import numpy as np

from .mrtlb import Config
from .simulation import Simulation


def amplification(s, rho, ux, uy, T, dx=1e-3, dy=1e-3, dt=1e-5, n=128, axis=0, version=1,
                  modified=True, eps=1e-6, device="cuda"):
    """Returns (k d for m = 0..n/2, G of shape (n/2 + 1, 16, 16), complex)."""
    nx, ny = (n, 1) if axis == 0 else (1, n)
    cfg = Config(nx=nx, ny=ny, dx=dx, dy=dy, dt=dt, s=tuple(float(v) for v in s),
                 bc=(("periodic", 0, 0, 1),) * 4, eq_version=version, modified=modified, precision="fp64")
    one = np.ones((ny, nx))
    cols = []
    with Simulation(cfg, device=device) as sim:
        sim.init_equilibrium(rho * one, ux * one, uy * one, T * one)
        f0 = sim.get_f()
        for q in range(16):
            resp = []
            for sign in (1.0, -1.0):
                f = f0.copy()
                f[q, 0, 0] += sign * eps
                sim.set_f(f)
                sim.step(1)
                resp.append(sim.get_f())
            r = (resp[0] - resp[1]) / (2.0 * eps)            # (16, ny, nx)
            r = r[:, 0, :] if axis == 0 else r[:, :, 0]      # along the axis
            cols.append(np.fft.fft(r, axis=1)[:, : n // 2 + 1])
    G = np.stack(cols, axis=1)                                 # (16, 16, m)
    kd = 2.0 * np.pi * np.arange(n // 2 + 1) / n
    return kd, np.moveaxis(G, 2, 0)


def max_growth(s, rho, ux, uy, T, **kw):
    """max over k of the largest eigenvalue modulus of G(k)."""
    _, G = amplification(s, rho, ux, uy, T, **kw)
    return float(max(np.abs(np.linalg.eigvals(g)).max() for g in G))
