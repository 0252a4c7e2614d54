"""Batched stepping (many uneven grids, one launch per step, CUDA graphs,
autotuned tiles) against the same instances stepped one by one, and against
the FP64 oracle."""
import numpy as np
import pytest

from oracle import equilibrium as oeq
from oracle import fdlb
from paper_1106_0785_gb300 import mrtlb as M
from paper_1106_0785_gb300 import workloads
from paper_1106_0785_gb300.simulation import Batch, Simulation

pytestmark = pytest.mark.gpu


def _instances(precision):
    """Six small instances: Sod-type tubes, Couette channels (NEE walls) and
    an interface-with-shock grid, of uneven shapes with ragged strips."""
    out = []
    for nx, ny, right in ((300, 5, (0.125, 0.8)), (150, 9, (0.2, 2.0)), (257, 40, (0.5, 1.5))):
        out.append(workloads.sod(nx=nx, ny=ny, precision=precision, right=right))
    for nx, ny, Pr, U in ((130, 12, 0.5, 0.4), (257, 7, 2.0, 0.8), (64, 33, 1.3, 0.2)):
        out.append(workloads.couette(Pr=Pr, nx=nx, ny=ny, precision=precision, U=U))
    out.append(workloads.richtmyer_meshkov(nx=200, ny=36, precision=precision))
    # the boundary kinds of Sec. IV B and IV A: inflow, outflow and reflecting
    # sides (a small shock-bubble grid) and diffuse-reflection walls
    cfg, fields = workloads.shock_bubble(nx=600, ny=30, precision=precision, radius=10.0)
    out.append((cfg, fields))
    out.append(workloads.slip_couette(nx=100, ny=5, precision=precision))
    # per-instance models: equilibrium versions 3 and 2, and one instance
    # without the energy-flux modification
    out[2][0].eq_version = 3
    out[3][0].modified = False
    out[4][0].eq_version = 2
    return out


def _sims(insts, kernel=None):
    sims = []
    for cfg, fields in insts:
        s = Simulation(cfg)
        if kernel is not None:
            s.set_kernel(kernel)
        s.init_equilibrium(*fields)
        sims.append(s)
    return sims


def _rel(a, b):
    scale = np.abs(b).reshape(16, -1).max(1)
    return (np.abs(a - b).reshape(16, -1).max(1) / scale).max()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_matches_instances_stepped_alone(cuda, precision):
    insts = _instances(precision)
    ref = _sims(insts, M.MRTLB_KERNEL_TILED)
    for s in ref:
        s.step(21)
    want = [s.get_f() for s in ref]
    sims = _sims(insts)
    with Batch(sims) as b:
        b.set_graph_steps(8)  # 2 graph replays, then 5 plain launches
        b.step(21)
        b.sync()
    for s, w in zip(sims, want):
        assert s.steps == 21
        got = s.get_f()
        assert _rel(got, w) < (1e-13 if precision == "fp64" else 1e-6)


def test_batch_fp64_matches_oracle(cuda):
    """Three instances with their own models (equilibrium version 3, no
    modification, version 2) in one batch, each against the oracle."""
    insts = _instances("fp64")[2:5]
    sims = _sims(insts)
    with Batch(sims) as b:
        b.step(12)
        b.sync()
    for (cfg, (rho, ux, uy, T)), s in zip(insts, sims):
        sides = tuple(fdlb.Side({"periodic": fdlb.PERIODIC, "outflow": fdlb.OUTFLOW,
                                 "wall": fdlb.WALL}[k], a, c, t) for k, a, c, t in cfg.bc)
        p = fdlb.Params(nx=cfg.nx, ny=cfg.ny, dx=cfg.dx, dy=cfg.dy, dt=cfg.dt, s=np.asarray(cfg.s),
                        sides=sides, version=cfg.eq_version, modified=cfg.modified)
        ref = fdlb.run(fdlb.prepare(oeq.feq(rho, ux, uy, T, version=cfg.eq_version), p), p, 12)
        assert _rel(s.get_f(), ref) < 1e-11


def test_tile_shapes_give_identical_results(cuda):
    insts = _instances("fp32")
    res = []
    for bx, sl in ((128, 32), (64, 8), (128, 5)):
        sims = _sims(insts)
        with Batch(sims) as b:
            b.set_tiles(bx, sl)
            assert b.tiles[:2] == (bx, sl)
            b.step(9)
            b.sync()
        res.append([s.get_f() for s in sims])
    for other in res[1:]:
        for a, c in zip(res[0], other):
            assert np.array_equal(a, c)  # the per-node arithmetic does not depend on the tiling


def test_tune_restores_state_and_uses_its_cache(cuda, tmp_path):
    insts = _instances("fp32")
    sims = _sims(insts)
    before = [s.get_f() for s in sims]
    cache = str(tmp_path / "tune.txt")
    with Batch(sims) as b:
        bx, sl = b.tune(cache, trial_steps=3)
        assert b.tiles[:2] == (bx, sl)
        after = [s.get_f() for s in sims]
        for x, y in zip(before, after):
            assert np.array_equal(x, y)
        lines = open(cache).read().split("\n")
        assert len([ln for ln in lines if ln.strip()]) == 1
        assert b.tune(cache, trial_steps=3) == (bx, sl)  # cache hit
        assert len([ln for ln in open(cache).read().split("\n") if ln.strip()]) == 1
        b.step(4)
        b.sync()


def test_batch_requires_matching_instances(cuda):
    a, _ = workloads.sod(nx=130, ny=5, precision="fp32")
    c, _ = workloads.sod(nx=130, ny=5, precision="fp64")
    s1, s2 = Simulation(a), Simulation(c)
    with pytest.raises(M.MrtlbError):
        Batch([s1, s2])
    s3 = Simulation(a)
    s3.step(1)
    with pytest.raises(M.MrtlbError):
        Batch([s1, s3])  # different buffer parity
    with Batch([s1, Simulation(a)]) as b:
        s1.step(1)  # stepped outside the batch
        with pytest.raises(M.MrtlbError) as ei:
            b.step(1)
        assert ei.value.code == M.MRTLB_ERR_STATE


def test_batch_refuses_an_instance_bound_to_other_buffers(cuda):
    """The batch's tables hold each instance's state buffers: binding an
    instance to new buffers afterwards (which also resets its parity to the
    batch's) makes the next batched step refuse rather than write through
    the old pointers."""
    import torch
    a, fields = workloads.sod(nx=130, ny=5, precision="fp32")
    s1, s2 = Simulation(a), Simulation(a)
    for s in (s1, s2):
        s.init_equilibrium(*fields)
    with Batch([s1, s2]) as b:
        b.step(2)
        b.sync()
        new = [torch.empty(s1.state_bytes, dtype=torch.uint8, device=cuda) for _ in range(2)]
        M.mrtlb_bind(s1.ctx, new[0], new[1], s1.state_bytes)
        s1.buffers = new
        with pytest.raises(M.MrtlbError) as ei:
            b.step(1)
        assert ei.value.code == M.MRTLB_ERR_STATE


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_follows_rates_set_on_an_instance(cuda, precision):
    """The batch's tables hold each instance's coefficient blocks: rates set
    on an instance with mrtlb_set_rates after the batch was made (here on a
    Couette channel with walls, whose wall table holds them too) take effect
    at the next batched step, inside the captured time loop, as they do for
    the instance stepped alone."""
    insts = [workloads.sod(nx=300, ny=5, precision=precision),
             workloads.couette(Pr=0.5, nx=130, ny=12, precision=precision, U=0.4)]
    ref = _sims(insts, M.MRTLB_KERNEL_TILED)
    sims = _sims(insts)
    for s in ref:
        s.step(13)
    with Batch(sims) as b:
        b.set_graph_steps(8)
        b.step(13)
        b.sync()
        for group in (ref, sims):
            s = np.array(group[1].rates())
            s[6:8] *= 4.0  # Pr 0.5 -> 2 (s7, s8)
            s[4:6] *= 0.5
            group[1].set_rates(s)
        for s in ref:
            s.step(19)
        b.step(19)
        b.sync()
    for s, r in zip(sims, ref):
        assert _rel(s.get_f(), r.get_f()) < (1e-13 if precision == "fp64" else 1e-6)
    # and the change matters: the channel stepped without it differs
    other = _sims(insts[1:], M.MRTLB_KERNEL_TILED)[0]
    other.step(32)
    assert _rel(other.get_f(), ref[1].get_f()) > 1e-6


def test_batch_reports_a_nonphysical_instance(cuda):
    """A negative temperature in one instance's input makes the batched step
    latch the non-physical flag, which mrtlb_batch_sync reports
    (MRTLB_ERR_NONPHYSICAL); the other instance is left as it was stepped."""
    a, fa = workloads.sod(nx=130, ny=5, precision="fp32")
    rho, ux, uy, T = (np.array(x, copy=True) for x in fa)
    T[2, 40] = -0.5
    s1, s2 = Simulation(a), Simulation(a)
    s1.init_equilibrium(*fa)
    s2.init_equilibrium(rho, ux, uy, T)
    with Batch([s1, s2]) as b:
        b.step(2)
        with pytest.raises(M.MrtlbError) as e:
            b.sync()
        assert e.value.code == M.MRTLB_ERR_NONPHYSICAL
    ref = Simulation(a)
    ref.set_kernel(M.MRTLB_KERNEL_TILED)
    ref.init_equilibrium(*fa)
    ref.step(2)
    assert _rel(s1.get_f(), ref.get_f()) < 1e-6


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("bc", ["periodic", "outflow_xy", "walls_y", "reflect_y", "diffuse_x", "inflow"])
def test_batch_of_degenerate_grids(cuda, bc, precision):
    """Degenerate grids batched together (a single node, single rows and
    columns, grids narrower than a column strip or shorter than a row
    segment, and one ordinary grid beside them), 3 batched steps, each
    instance against the oracle (FP64 1e-11 per plane; FP32 from the
    FP32-rounded start, 2e-6 of the state's scale)."""
    from test_gpu_parity import BCS, _cfg, _input, oracle_params, rel_plane_err
    shapes = [(1, 1), (2, 3), (1, 6), (7, 1), (3, 130), (129, 2), (300, 5)]
    cases = []
    for nx, ny in shapes:
        if bc == "walls_y" and ny < 3:  # (walls need three nodes across)
            continue
        cfg = _cfg(nx, ny, BCS[bc], precision)
        (rho, ux, uy, T), nz = _input(cfg, 40 + nx + ny)
        p = oracle_params(cfg)
        f0 = fdlb.prepare(oeq.feq(rho, ux, uy, T) + nz, p)
        if precision == "fp32":
            f0 = f0.astype(np.float32).astype(np.float64)
        s = Simulation(cfg)
        s.set_f(f0.astype(np.float32) if precision == "fp32" else f0)
        cases.append((s, p, f0))
    with Batch([c[0] for c in cases]) as b:
        b.step(3)
        b.sync()
    for s, p, f0 in cases:
        g = s.get_f()
        s.close()
        assert np.isfinite(g).all()
        f = fdlb.run(f0, p, 3)
        if precision == "fp64":
            assert rel_plane_err(g, f) < 1e-11
        else:  # against the state's scale: FP32 rounds at the scale of the moments, and a
            # single node's fast planes (0.004) can be 50x smaller than its largest (0.2)
            assert np.abs(g - f).max() < 2e-6 * np.abs(f).max()
