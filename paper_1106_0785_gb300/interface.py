"""Differentiable initial fields of the Richtmyer-Meshkov set-up and its
mixing width, in torch (for gradients with respect to the interface shape).

Same recipe as workloads.richtmyer_meshkov: light gas (rho 1) | heavy gas
(rho 3) at p = 1 across x_I(y) = x_iface + sum_k a_k cos(2 pi k y / Ly),
tanh-smoothed over 3 cells, with a Mach-`mach` shock (gamma = 2 normal-shock
state) at x_shock moving into the light gas.  The mixing width,
W = dx dy sum_ij (rho_ij - mean_j rho_ij)^2, is zero for a flat interface
and grows with its distortion.
"""
import math

import torch

from .workloads import normal_shock


def rm_initial_fields(amplitudes, nx, ny, mach=1.5, rho_light=1.0, rho_heavy=3.0, x_iface=0.5,
                      x_shock=0.3, device=None):
    """(rho, ux, uy, T) as FP64 tensors [ny][nx], differentiable in amplitudes."""
    a = amplitudes.to(device=device, dtype=torch.float64)
    dx = 1.0 / nx
    Ly = ny * dx
    x = (torch.arange(nx, dtype=torch.float64, device=device) + 0.5) * dx
    y = (torch.arange(ny, dtype=torch.float64, device=device) + 0.5) * dx
    k = torch.arange(1, a.numel() + 1, dtype=torch.float64, device=device)
    xi = x_iface + (a[None, :] * torch.cos(2.0 * math.pi * k[None, :] * y[:, None] / Ly)).sum(1)
    w = 0.5 * (1.0 + torch.tanh((x[None, :] - xi[:, None]) / (3.0 * dx)))
    rho = rho_light + (rho_heavy - rho_light) * w
    rho2, u2, p2, _ = normal_shock(rho_light, 1.0, mach)
    s = 1.0 - 0.5 * (1.0 + torch.tanh((x[None, :] - x_shock) / (2.0 * dx)))
    s = s.expand(ny, nx)
    rho = rho + (rho2 - rho_light) * s
    p = 1.0 + (p2 - 1.0) * s
    ux = u2 * s
    return rho, ux.contiguous(), torch.zeros_like(rho), (p / rho)


def mixing_width(rho, dx, dy):
    """W = dx dy sum (rho - its y-average per x column)^2 for rho [ny][nx]."""
    return dx * dy * ((rho - rho.mean(dim=0, keepdim=True)) ** 2).sum()
