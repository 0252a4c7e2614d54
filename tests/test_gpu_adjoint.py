"""The hand-written adjoint against the FP64 oracle's exact tangent.

For random directions v (on the initial state) and w (on the final state),
<w, J v> from a complex-step derivative of the oracle's steps must equal
<J^T w, v> from the CUDA adjoint (FP64 path), and the rate gradients must
equal <w, dF/ds_k> from complex steps in s_k.  These dot-product tests pin
every term of the transpose: Lax-Wendroff, collision, the modification's
local and neighbour terms, ghosts and NEE walls, and the checkpointed
multi-step recompute.
"""
import numpy as np
import pytest

from oracle import equilibrium as oeq
from oracle import fdlb
from paper_1106_0785_gb300 import mrtlb as M
from paper_1106_0785_gb300 import workloads
from paper_1106_0785_gb300.simulation import Simulation

pytestmark = pytest.mark.gpu

H = 1e-30

BCS = {
    "periodic": (("periodic", 0, 0, 1),) * 4,
    "outflow_x": (("outflow", 0, 0, 1),) * 2 + (("periodic", 0, 0, 1),) * 2,
    "walls_y": (("periodic", 0, 0, 1),) * 2 + (("wall", 0.1, 0.0, 1.1), ("wall", 0.5, -0.05, 0.95)),
    "walls_x": (("wall", 0.02, 0.3, 1.0), ("wall", 0.0, -0.2, 1.2)) + (("outflow", 0, 0, 1),) * 2,
    "reflect": (("reflect", 0, 0, 1),) * 2 + (("reflect", 0, 0, 1),) * 2,
    "inflow": (("outflow", 0, 0, 1), ("inflow", -0.05, 0.02, 1.1, 1.2)) + (("reflect", 0, 0, 1),) * 2,
    "diffuse": (("periodic", 0, 0, 1),) * 2 + (("diffuse", -0.1, 0.02, 1.0), ("diffuse", 0.1, 0.0, 1.1)),
}


def _cfg(nx, ny, bc, version=1, precision="fp64"):
    s = np.random.default_rng(5).uniform(50, 2000, 16)
    s[:4] = 0
    return M.Config(nx=nx, ny=ny, dx=0.01, dy=0.011, dt=2e-4, s=tuple(s), bc=bc,
                    eq_version=version, precision=precision)


KINDS = {"periodic": fdlb.PERIODIC, "outflow": fdlb.OUTFLOW, "wall": fdlb.WALL,
         "inflow": fdlb.INFLOW, "reflect": fdlb.REFLECT, "diffuse": fdlb.DIFFUSE}


def _oracle_params(cfg, s=None):
    sides = tuple(fdlb.Side(KINDS[side[0]], *side[1:]) for side in cfg.bc)
    p = fdlb.Params(nx=cfg.nx, ny=cfg.ny, dx=cfg.dx, dy=cfg.dy, dt=cfg.dt, s=np.asarray(cfg.s),
                    sides=sides, version=cfg.eq_version, modified=cfg.modified)
    if s is not None:
        p.s = s
    return p


def _state(cfg, seed):
    rho, ux, uy, T = workloads.smooth_fields(cfg.nx, cfg.ny, seed)
    f0 = oeq.feq(rho, ux, uy, T, cfg.eq_version) + workloads.noise((16, cfg.ny, cfg.nx), seed + 1, 1e-3)
    return fdlb.prepare(f0, _oracle_params(cfg))


KERNELS = {"plain": M.MRTLB_KERNEL_PLAIN, "tiled": M.MRTLB_KERNEL_TILED}


def _adjoint(cuda, cfg, f0, K, w=None, seed_macros=None, interval=None, kernel="auto"):
    """The tiled kernel choice runs the adjoint as the fused row march, the
    plain one as the two-pass gather."""
    import torch
    with Simulation(cfg) as sim:
        if kernel != "auto":
            sim.set_kernel(KERNELS[kernel])
        sim.set_f(f0)
        sim.adjoint_forward(K, interval)
        dm = None if seed_macros is None else torch.from_numpy(seed_macros).to(cuda)
        dw = None if w is None else torch.from_numpy(w).to(cuda)
        ds, df0 = sim.adjoint_backward(dL_dmacros=dm, dL_dfK=dw)
        return ds, df0.cpu().numpy()


@pytest.mark.parametrize("kernel", list(KERNELS))
@pytest.mark.parametrize("bc", list(BCS))
@pytest.mark.parametrize("version", [1, 2, 3])
def test_one_step_adjoint_dot_product(cuda, bc, version, kernel):
    cfg = _cfg(140, 21, BCS[bc], version)
    f0 = _state(cfg, 100)
    rng = np.random.default_rng(101)
    v = rng.standard_normal(f0.shape)
    w = rng.standard_normal(f0.shape)
    ds, lam0 = _adjoint(cuda, cfg, f0, 1, w=w, kernel=kernel)
    p = _oracle_params(cfg)
    Jv = fdlb.step(f0 + 1j * H * v, p).imag / H
    lhs, rhs = float((w * Jv).sum()), float((lam0 * v).sum())
    assert abs(lhs - rhs) < 1e-11 * np.abs(w * Jv).sum(), (lhs, rhs)
    # rate gradients: <w, dF/ds_k>
    for k in range(4, 16):
        sk = np.asarray(cfg.s, dtype=complex)
        sk[k] += 1j * H
        dF = fdlb.step(f0.astype(complex), _oracle_params(cfg, sk)).imag / H
        ref = float((w * dF).sum())
        assert abs(ds[k] - ref) < 1e-10 * np.abs(w * dF).sum(), (k, ds[k], ref)
    assert np.all(ds[:4] == 0)


@pytest.mark.parametrize("kernel", list(KERNELS))
@pytest.mark.parametrize("interval", [3, 0])
def test_multi_step_adjoint_through_checkpoints(cuda, interval, kernel):
    """K = 7: segments 3 + 3 + 1 (the first two recomputed from checkpoints),
    or all 7 states kept (automatic choice on a small grid)."""
    cfg = _cfg(70, 13, BCS["walls_y"])
    f0 = _state(cfg, 110)
    rng = np.random.default_rng(111)
    v = rng.standard_normal(f0.shape)
    w = rng.standard_normal(f0.shape)
    ds, lam0 = _adjoint(cuda, cfg, f0, 7, w=w, interval=interval, kernel=kernel)
    p = _oracle_params(cfg)
    Jv = fdlb.run(f0 + 1j * H * v, p, 7).imag / H
    lhs, rhs = float((w * Jv).sum()), float((lam0 * v).sum())
    assert abs(lhs - rhs) < 1e-10 * np.abs(w * Jv).sum()
    k = 6
    sk = np.asarray(cfg.s, dtype=complex)
    sk[k] += 1j * H
    dF = fdlb.run(f0.astype(complex), _oracle_params(cfg, sk), 7).imag / H
    assert abs(ds[k] - float((w * dF).sum())) < 1e-9 * np.abs(w * dF).sum()


@pytest.mark.parametrize("kernel", list(KERNELS))
def test_macro_seed(cuda, kernel):
    """L = sum(a rho + b ux + c uy + d T) of the final macroscopic fields."""
    cfg = _cfg(66, 17, BCS["outflow_x"])
    f0 = _state(cfg, 120)
    rng = np.random.default_rng(121)
    weights = rng.standard_normal((4, cfg.ny, cfg.nx))
    v = rng.standard_normal(f0.shape)
    ds, lam0 = _adjoint(cuda, cfg, f0, 4, seed_macros=weights, kernel=kernel)
    p = _oracle_params(cfg)
    fK = fdlb.run(f0 + 1j * H * v, p, 4)
    dL = float(sum((weights[k] * m).sum() for k, m in enumerate(fdlb.macros(fK))).imag / H)
    assert abs(dL - float((lam0 * v).sum())) < 1e-10 * np.abs(weights).sum()


@pytest.mark.parametrize("version", [1, 2, 3])
def test_equilibrium_adjoint(cuda, version):
    import torch
    cfg = _cfg(50, 9, BCS["periodic"], version=version)
    rho, ux, uy, T = workloads.smooth_fields(cfg.nx, cfg.ny, 130)
    rng = np.random.default_rng(131)
    lam = rng.standard_normal((16, cfg.ny, cfg.nx))
    d = [rng.standard_normal((cfg.ny, cfg.nx)) for _ in range(4)]
    with Simulation(cfg) as sim:
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(cuda)
        outs = sim.equilibrium_adjoint(t(lam), t(rho), t(ux), t(uy), t(T))
    rhs = sum(float((o.cpu().numpy() * di).sum()) for o, di in zip(outs, d))
    jf = oeq.feq(rho + 1j * H * d[0], ux + 1j * H * d[1], uy + 1j * H * d[2], T + 1j * H * d[3], version).imag / H
    lhs = float((lam * jf).sum())
    assert abs(lhs - rhs) < 1e-11 * np.abs(lam * jf).sum()


@pytest.mark.parametrize("kernel", list(KERNELS))
def test_fp32_adjoint_close_to_fp64(cuda, kernel):
    cfg64 = _cfg(140, 21, BCS["walls_y"])
    f0 = _state(cfg64, 140)
    w = np.random.default_rng(141).standard_normal(f0.shape)
    ds64, l64 = _adjoint(cuda, cfg64, f0, 5, w=w)
    cfg32 = _cfg(140, 21, BCS["walls_y"], precision="fp32")
    ds32, l32 = _adjoint(cuda, cfg32, f0.astype(np.float32), 5, w=w, kernel=kernel)
    assert np.abs(l32 - l64).max() < 1e-4 * np.abs(l64).max()
    assert np.allclose(ds32[4:], ds64[4:], rtol=1e-3, atol=1e-4 * np.abs(ds64).max())


@pytest.mark.parametrize("interval", [2, 0])
def test_backward_twice_after_one_forward(cuda, interval):
    """A second backward pass with another seed after the same forward pass
    must see the same states (the slots are refilled from checkpoints), on
    the tiled step kernel (grid wide enough for it)."""
    import torch
    cfg = _cfg(300, 40, BCS["outflow_x"])
    f0 = _state(cfg, 150)
    rng = np.random.default_rng(151)
    w1, w2 = rng.standard_normal(f0.shape), rng.standard_normal(f0.shape)
    with Simulation(cfg) as sim:
        sim.set_kernel(M.MRTLB_KERNEL_TILED)
        sim.set_f(f0)
        sim.adjoint_forward(5, interval)
        fK = sim.get_f()
        res = [sim.adjoint_backward(dL_dfK=torch.from_numpy(w).to(cuda)) for w in (w1, w2, w1)]
    assert np.allclose(fK, fdlb.run(f0, _oracle_params(cfg), 5), rtol=0, atol=1e-12)
    l1, l2, l3 = (r[1].cpu().numpy() for r in res)
    assert np.array_equal(l1, l3)
    # (the rate gradients are sums of FP64 atomics: equal up to their order)
    assert np.allclose(res[0][0], res[2][0], rtol=1e-12, atol=0)
    v = rng.standard_normal(f0.shape)
    Jv = fdlb.run(f0 + 1j * H * v, _oracle_params(cfg), 5).imag / H
    for w, lam in ((w1, l1), (w2, l2)):
        lhs, rhs = float((w * Jv).sum()), float((lam * v).sum())
        assert abs(lhs - rhs) < 1e-10 * np.abs(w * Jv).sum()


def test_march_matches_two_pass_on_a_ragged_grid(cuda):
    """FP32, 1030 x 260 (ragged strips and row segments), 3 steps: the fused
    row march and the two-pass gather give the same adjoint."""
    import torch
    cfg = _cfg(1030, 260, BCS["walls_x"], precision="fp32")
    f0 = _state(_cfg(1030, 260, BCS["walls_x"]), 160).astype(np.float32)
    w = np.random.default_rng(161).standard_normal(f0.shape)
    res = {}
    for kernel in KERNELS:
        with Simulation(cfg) as sim:
            sim.set_kernel(KERNELS[kernel])
            sim.set_f(f0)
            sim.adjoint_forward(3)
            res[kernel] = sim.adjoint_backward(dL_dfK=torch.from_numpy(w).to(cuda))
    (dp, lp), (dt, lt) = res["plain"], res["tiled"]
    lp, lt = lp.cpu().numpy(), lt.cpu().numpy()
    assert np.abs(lp - lt).max() < 1e-5 * np.abs(lp).max()
    assert np.allclose(dp[4:], dt[4:], rtol=1e-4, atol=1e-6 * np.abs(dp).max())


@pytest.mark.parametrize("kernel", list(KERNELS))
def test_repeated_passes_reuse_the_adjoint_state(cuda, kernel):
    """A second forward pass of the same length reuses the stored states'
    buffers and plans and gives the same adjoint; a pass of another length
    re-plans and matches a fresh context."""
    import torch
    cfg = _cfg(300, 40, BCS["inflow"])
    f0 = _state(cfg, 170)
    w = torch.from_numpy(np.random.default_rng(171).standard_normal(f0.shape)).to(cuda)

    def run(sim, K):
        sim.set_f(f0)
        sim.adjoint_forward(K)
        return sim.adjoint_backward(dL_dfK=w)

    with Simulation(cfg) as sim:
        sim.set_kernel(KERNELS[kernel])
        (d1, l1), (d2, l2), (d3, l3) = run(sim, 5), run(sim, 5), run(sim, 9)
    with Simulation(cfg) as fresh:
        fresh.set_kernel(KERNELS[kernel])
        d4, l4 = run(fresh, 9)
    assert np.array_equal(l1.cpu().numpy(), l2.cpu().numpy())
    assert np.allclose(d1, d2, rtol=1e-12, atol=0)
    assert np.array_equal(l3.cpu().numpy(), l4.cpu().numpy())
    assert np.allclose(d3, d4, rtol=1e-12, atol=0)


@pytest.mark.parametrize("change", ["step", "set_f", "set_rates", "init_equilibrium", "forward_again"])
def test_backward_refuses_a_changed_context(cuda, change):
    """A backward pass differentiates the forward pass it follows: any call
    that changed the state or the rates in between makes it refuse
    (MRTLB_ERR_STATE) rather than mix two runs; an unchanged context still
    gives the same gradients."""
    import torch
    cfg = _cfg(40, 12, BCS["periodic"])
    f0 = _state(cfg, 50)
    w = torch.from_numpy(workloads.noise((16, cfg.ny, cfg.nx), 51)).to(cuda)
    with Simulation(cfg) as sim:
        sim.set_f(f0)
        sim.adjoint_forward(3)
        p1 = sim.adjoint_pass()
        assert p1 > 0
        ds1, _ = sim.adjoint_backward(dL_dfK=w)
        rho, ux, uy, T = workloads.smooth_fields(cfg.nx, cfg.ny, 52)
        if change == "step":
            sim.step(1)
        elif change == "set_f":
            sim.set_f(f0)
        elif change == "set_rates":
            sim.set_rates(np.asarray(cfg.s))
        elif change == "init_equilibrium":
            sim.init_equilibrium(rho, ux, uy, T)
        else:
            sim.set_f(f0)
            sim.adjoint_forward(3)
            assert sim.adjoint_pass() == p1 + 1
            ds2, _ = sim.adjoint_backward(dL_dfK=w)
            assert np.allclose(ds2, ds1, rtol=1e-12, atol=0)
            return
        assert sim.adjoint_pass() == 0
        with pytest.raises(M.MrtlbError) as e:
            sim.adjoint_backward(dL_dfK=w)
        assert e.value.code == M.MRTLB_ERR_STATE


def test_autograd_refuses_an_overwritten_run(cuda):
    """Two runs on one Simulation before backward: the first one's backward
    raises (its checkpoints are gone), the second one's works."""
    import torch
    from paper_1106_0785_gb300 import autograd
    cfg = _cfg(40, 12, BCS["periodic"])
    rho, ux, uy, T = (torch.from_numpy(a).to(cuda) for a in workloads.smooth_fields(cfg.nx, cfg.ny, 53))
    s = torch.tensor(cfg.s, dtype=torch.float64, requires_grad=True)
    with Simulation(cfg) as sim:
        out1 = autograd.run(sim, rho, ux, uy, T, s, 2)
        out2 = autograd.run(sim, rho, ux, uy, T, s, 3)
        out2[3].sum().backward(retain_graph=True)
        assert torch.isfinite(s.grad).all()
        with pytest.raises(RuntimeError, match="run or changed after this forward pass"):
            out1[3].sum().backward()


@pytest.mark.parametrize("kernel", list(KERNELS))
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_backward_without_rate_gradients(cuda, kernel, precision):
    """dL_ds = NULL skips the rate gradients' work in the adjoint steps; the
    state adjoint dL/df0 is the same as with them, to the rounding of the
    precision (the two kernel variants are compiled separately, so their
    multiply-adds may contract differently)."""
    import torch
    cfg = _cfg(150, 37, BCS["walls_y"], precision=precision)
    f0 = _state(cfg, 70)
    if precision == "fp32":
        f0 = f0.astype(np.float32)
    w = torch.from_numpy(workloads.noise((16, cfg.ny, cfg.nx), 71)).to(cuda)
    with Simulation(cfg) as sim:
        sim.set_kernel(KERNELS[kernel])
        sim.set_f(f0)
        sim.adjoint_forward(4, interval=2)
        ds, d1 = sim.adjoint_backward(dL_dfK=w)
        none, d2 = sim.adjoint_backward(dL_dfK=w, want_ds=False)
    assert none is None and np.abs(ds[4:]).max() > 0
    a, b = d1.cpu().numpy(), d2.cpu().numpy()
    scale = np.abs(a).reshape(16, -1).max(1)
    tol = 1e-12 if precision == "fp64" else 1e-5
    assert (np.abs(b - a).reshape(16, -1).max(1) / scale).max() < tol


def test_forward_pass_that_cannot_allocate_keeps_nothing(cuda):
    """A forward pass whose segment of states cannot be allocated (segments
    of a million states: about 2 TB here, far beyond the device) fails with
    MRTLB_ERR_CUDA after its checkpoints were allocated and before any step
    runs, and keeps nothing: no backward pass is possible, the same request
    fails the same way again (instead of reusing the half-built buffers),
    and a pass that fits then gives what a fresh context gives."""
    import torch
    cfg = _cfg(300, 40, BCS["outflow_x"])
    f0 = _state(cfg, 180)
    w = torch.from_numpy(np.random.default_rng(181).standard_normal(f0.shape)).to(cuda)
    with Simulation(cfg) as sim:
        sim.set_f(f0)
        for _ in range(2):
            with pytest.raises(M.MrtlbError) as e:
                sim.adjoint_forward(2_000_000, interval=1_000_000)
            assert e.value.code == M.MRTLB_ERR_CUDA
            assert sim.adjoint_pass() == 0
            assert sim.steps == 0
        with pytest.raises(M.MrtlbError) as e:
            sim.adjoint_backward(dL_dfK=w)
        assert e.value.code == M.MRTLB_ERR_STATE
        sim.adjoint_forward(5, interval=0)
        _, l1 = sim.adjoint_backward(dL_dfK=w)
    with Simulation(cfg) as fresh:
        fresh.set_f(f0)
        fresh.adjoint_forward(5)
        _, l2 = fresh.adjoint_backward(dL_dfK=w)
    assert np.array_equal(l1.cpu().numpy(), l2.cpu().numpy())


def test_backward_reports_a_nonphysical_forward_pass(cuda):
    """A forward pass from a state with a negative temperature at one node
    meets a non-physical state; the backward pass reports it
    (MRTLB_ERR_NONPHYSICAL) instead of returning gradients of that run."""
    import torch
    cfg = _cfg(64, 8, BCS["periodic"], precision="fp32")
    rho, ux, uy, T = workloads.smooth_fields(cfg.nx, cfg.ny, 190)
    T[3, 5] = -0.5
    seed = torch.zeros((4, cfg.ny, cfg.nx), dtype=torch.float64, device=cuda)
    seed[3] = 1.0
    with Simulation(cfg) as sim:
        sim.init_equilibrium(rho, ux, uy, T)
        sim.adjoint_forward(3)
        with pytest.raises(M.MrtlbError) as e:
            sim.adjoint_backward(dL_dmacros=seed)
        assert e.value.code == M.MRTLB_ERR_NONPHYSICAL


@pytest.mark.parametrize("kernel", list(KERNELS))
@pytest.mark.parametrize("shape", [(1, 1), (2, 3), (1, 6), (7, 1), (3, 130), (129, 2)], ids=lambda s: "%dx%d" % s)
@pytest.mark.parametrize("bc", ["periodic", "outflow_x", "walls_y", "reflect", "inflow", "diffuse"])
def test_adjoint_dot_product_on_degenerate_grids(cuda, bc, shape, kernel):
    """Two adjoint steps on degenerate grids (a single node, single rows and
    columns, grids narrower than a column strip or shorter than a row
    segment) through both adjoint kernels: <w, Jv> = <J^T w, v> against the
    oracle's complex-step tangent (FP64)."""
    nx, ny = shape
    cfg = _cfg(nx, ny, BCS[bc])
    if bc == "walls_y" and ny < 3:  # (walls need three nodes across)
        with pytest.raises(M.MrtlbError):
            Simulation(cfg)
        return
    f0 = _state(cfg, 200 + nx + ny)
    rng = np.random.default_rng(201)
    v = rng.standard_normal(f0.shape)
    w = rng.standard_normal(f0.shape)
    _, lam0 = _adjoint(cuda, cfg, f0, 2, w=w, kernel=kernel)
    Jv = fdlb.run(f0 + 1j * H * v, _oracle_params(cfg), 2).imag / H
    lhs, rhs = float((w * Jv).sum()), float((lam0 * v).sum())
    assert abs(lhs - rhs) < 1e-11 * np.abs(w * Jv).sum(), (lhs, rhs)
