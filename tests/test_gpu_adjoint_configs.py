"""Gradients on the paper's workloads, FP32 forward + adjoint with sqrt(K)
checkpointing, against FP64 central finite differences (and the oracle's
own tangent for the Couette case).

(a) Thermal Couette flow 4 x 200, K = 5000 steps, loss sum (T - T_target)^2
    with T_target the closed form at Pr = 0.7, gradient with respect to the
    tied momentum rates s5 = s6 and energy-flux rates s7 = s8.
(b) Richtmyer-Meshkov 512 x 128, K = 800 steps, gradient of the interface
    mixing width with respect to 8 cosine amplitudes of the interface.
"""
import numpy as np
import pytest

from oracle import couette as ocouette
from oracle import equilibrium as oeq
from oracle import fdlb
from paper_1106_0785_gb300 import mrtlb as M
from paper_1106_0785_gb300 import workloads
from paper_1106_0785_gb300.simulation import Simulation

pytestmark = pytest.mark.gpu

U = 0.8


def _couette(precision):
    cfg, fields = workloads.couette(Pr=1.0, nx=4, ny=200, precision=precision, dt=1e-4, U=U,
                                    s_visc=1e2)
    y = np.arange(cfg.ny) / (cfg.ny - 1)
    target = ocouette.temperature(y, 1.0, 1.0, U, 1.0, 0.7, True)  # Pr = 0.7
    return cfg, fields, np.broadcast_to(target[:, None], (cfg.ny, cfg.nx)).copy()


def _couette_loss(sim, fields, target, s, K):
    sim.set_rates(s)
    sim.init_equilibrium(*fields)
    sim.step(K)
    T = sim.macros()[3]
    return float(((T - target) ** 2).sum())


def test_couette_rate_gradients(cuda):
    import torch
    K = 5000
    cfg, fields, target = _couette("fp32")
    s0 = np.asarray(cfg.s, dtype=float)
    with Simulation(cfg) as sim:
        sim.set_rates(s0)
        sim.init_equilibrium(*fields)
        sim.adjoint_forward(K, interval=71)  # sqrt(K) checkpoints: 71 segments of 71 steps, 70 recomputed
        T = sim.macros()[3]
        seed = np.zeros((4, cfg.ny, cfg.nx))
        seed[3] = 2.0 * (T - target)
        ds, _ = sim.adjoint_backward(dL_dmacros=torch.from_numpy(seed).to(cuda), want_df0=False)
    g_visc, g_cond = ds[4] + ds[5], ds[6] + ds[7]

    # FP64 central differences on the GPU's FP64 path
    cfg64, fields64, _ = _couette("fp64")
    fd = []
    with Simulation(cfg64) as sim:
        for pair in ((4, 5), (6, 7)):
            h = 1e-6 * max(abs(s0[pair[0]]), 1.0)
            vals = []
            for sign in (1, -1):
                s = s0.copy()
                s[list(pair)] += sign * h
                vals.append(_couette_loss(sim, fields64, target, s, K))
            fd.append((vals[0] - vals[1]) / (2 * h))
    assert np.isclose(g_visc, fd[0], rtol=2e-3), (g_visc, fd[0])
    assert np.isclose(g_cond, fd[1], rtol=2e-3), (g_cond, fd[1])

    # the oracle's own tangent (complex step in the tied rates), FP64
    sides = tuple(fdlb.Side({"periodic": fdlb.PERIODIC, "wall": fdlb.WALL}[k], a, b, t) for k, a, b, t in cfg.bc)
    rho, ux, uy, T0 = fields
    f0 = oeq.feq(rho, ux, uy, T0)
    for pair, g in (((4, 5), g_visc), ((6, 7), g_cond)):
        s = s0.astype(complex)
        s[list(pair)] += 1e-30j
        p = fdlb.Params(nx=cfg.nx, ny=cfg.ny, dx=cfg.dx, dy=cfg.dy, dt=cfg.dt, s=s0, sides=sides)
        p.s = s
        f = fdlb.run(fdlb.prepare(f0.astype(complex), p), p, K)
        Tk = fdlb.macros(f)[3]
        dL = float((2.0 * (Tk.real - target) * Tk.imag / 1e-30).sum())
        assert np.isclose(g, dL, rtol=2e-3), (g, dL)


def test_richtmyer_meshkov_interface_gradient(cuda):
    import torch

    from paper_1106_0785_gb300.autograd import run
    from paper_1106_0785_gb300.interface import mixing_width, rm_initial_fields

    K = 800
    nx, ny = 512, 128
    a0 = np.random.default_rng(0).uniform(0.0, 0.02, 8)

    def make(precision):
        cfg, _ = workloads.richtmyer_meshkov(nx=nx, ny=ny, precision=precision, dt=1.25e-4, x_shock=0.3,
                                             s_visc=4e3, s_cond=4e3, s_other=8e3)
        return cfg

    cfg = make("fp32")
    dx = cfg.dx
    with Simulation(cfg) as sim:
        M.mrtlb_adjoint_set_interval(sim.ctx, 29)  # sqrt(K) checkpoints: 28 segments of 29 steps, 27 recomputed
        a = torch.tensor(a0, dtype=torch.float64, device=cuda, requires_grad=True)
        s = torch.tensor(cfg.s, dtype=torch.float64)
        rho0, ux0, uy0, T0 = rm_initial_fields(a, nx, ny, x_shock=0.3, device=cuda)
        rho, _, _, _ = run(sim, rho0, ux0, uy0, T0, s, K)
        W = mixing_width(rho, dx, dx)
        W.backward()
        grad = a.grad.cpu().numpy()
        W0 = float(W.detach())

    cfg64 = make("fp64")
    fd = np.zeros(8)
    with Simulation(cfg64) as sim:
        def width(av):
            fields = rm_initial_fields(torch.tensor(av, dtype=torch.float64, device=cuda), nx, ny,
                                       x_shock=0.3, device=cuda)
            sim.init_equilibrium(*fields)
            sim.step(K)
            r = sim.macros(on_device=True)[0]
            return float(mixing_width(r, dx, dx))
        assert np.isclose(width(a0), W0, rtol=1e-5)
        for k in range(8):
            h = 1e-6
            e = np.zeros(8)
            e[k] = h
            fd[k] = (width(a0 + e) - width(a0 - e)) / (2 * h)
    assert np.allclose(grad, fd, rtol=5e-3, atol=5e-3 * np.abs(fd).max()), (grad, fd)
