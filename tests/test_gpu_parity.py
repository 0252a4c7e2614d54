"""CUDA path vs the FP64 oracle, through the C ABI.

Tolerances (fixed by the method's requirements for this implementation):
  FP64 path: 1e-12 of each plane's magnitude after one step from the same
             state (the step reorders sums and contracts multiply-adds, so it
             is not bitwise);
  FP32 path: 1e-5 relative in rho, u (normalised by max |u|) and T after 1000
             smooth-flow steps, 1e-4 relative L1 across shocks (and, on the
             bench's shocked crop, 1e-5 at every node after 1000 steps).
Grid sizes span several column strips (128 nodes in FP32, 64 in FP64) and
row segments, with ragged tails.
"""
import numpy as np
import pytest

from oracle import equilibrium as oeq
from oracle import fdlb
from paper_1106_0785_gb300 import mrtlb as M
from paper_1106_0785_gb300 import workloads
from paper_1106_0785_gb300.simulation import Simulation

pytestmark = pytest.mark.gpu

KERNELS = {"plain": M.MRTLB_KERNEL_PLAIN, "tiled": M.MRTLB_KERNEL_TILED}


KINDS = {"periodic": fdlb.PERIODIC, "outflow": fdlb.OUTFLOW, "wall": fdlb.WALL,
         "inflow": fdlb.INFLOW, "reflect": fdlb.REFLECT, "diffuse": fdlb.DIFFUSE}


def oracle_params(cfg):
    sides = []
    for side in cfg.bc:
        kind, ux, uy, T = side[:4]
        sides.append(fdlb.Side(KINDS[kind], ux, uy, T, *side[4:]))
    return fdlb.Params(nx=cfg.nx, ny=cfg.ny, dx=cfg.dx, dy=cfg.dy, dt=cfg.dt,
                       s=np.asarray(cfg.s), sides=tuple(sides), version=cfg.eq_version,
                       modified=cfg.modified)


def rel_plane_err(a, b):
    scale = np.abs(b).reshape(16, -1).max(1)
    return (np.abs(a - b).reshape(16, -1).max(1) / scale).max()


BCS = {
    "periodic": (("periodic", 0, 0, 1),) * 4,
    "outflow_x": (("outflow", 0, 0, 1),) * 2 + (("periodic", 0, 0, 1),) * 2,
    "outflow_xy": (("outflow", 0, 0, 1),) * 4,
    "walls_y": (("periodic", 0, 0, 1),) * 2 + (("wall", 0.1, 0.0, 1.1), ("wall", 0.5, -0.05, 0.95)),
    "walls_x": (("wall", 0.02, 0.3, 1.0), ("wall", 0.0, -0.2, 1.2)) + (("outflow", 0, 0, 1),) * 2,
    "reflect_y": (("periodic", 0, 0, 1),) * 2 + (("reflect", 0, 0, 1),) * 2,
    "reflect_x": (("reflect", 0, 0, 1),) * 2 + (("outflow", 0, 0, 1),) * 2,
    # the shock-bubble's sides: outflow left, fixed post-shock inflow right, reflecting top and bottom
    "inflow": (("outflow", 0, 0, 1), ("inflow", -0.05, 0.02, 1.1, 1.2)) + (("reflect", 0, 0, 1),) * 2,
    "diffuse_y": (("periodic", 0, 0, 1),) * 2 + (("diffuse", -0.1, 0.02, 1.0), ("diffuse", 0.1, 0.0, 1.1)),
    "diffuse_x": (("diffuse", 0.0, -0.2, 0.95), ("diffuse", 0.03, 0.2, 1.0)) + (("periodic", 0, 0, 1),) * 2,
}


def _cfg(nx, ny, bc, precision, version=1, modified=True, dt=2e-4, d=0.01):
    s = np.random.default_rng(5).uniform(50, 2000, 16)
    s[:4] = 0
    return M.Config(nx=nx, ny=ny, dx=d, dy=1.1 * d, dt=dt, s=tuple(s), bc=bc,
                    eq_version=version, modified=modified, precision=precision)


def _input(cfg, seed, noise=1e-3):
    rho, ux, uy, T = workloads.smooth_fields(cfg.nx, cfg.ny, seed)
    nz = workloads.noise((16, cfg.ny, cfg.nx), seed + 1, noise)
    return (rho, ux, uy, T), nz


@pytest.mark.parametrize("kernel", list(KERNELS))
@pytest.mark.parametrize("bc", list(BCS))
def test_fp64_one_step_parity(cuda, kernel, bc):
    cfg = _cfg(300, 70, BCS[bc], "fp64")
    (rho, ux, uy, T), nz = _input(cfg, 10)
    p = oracle_params(cfg)
    f0 = fdlb.prepare(oeq.feq(rho, ux, uy, T) + nz, p)
    with Simulation(cfg) as sim:
        sim.set_kernel(KERNELS[kernel])
        sim.set_f(f0)
        # get_f refills wall nodes (same values up to rounding)
        assert rel_plane_err(sim.get_f(), f0) < 1e-13
        sim.step(1)
        g1 = sim.get_f()
    f1 = fdlb.step(f0, p)
    assert rel_plane_err(g1, f1) < 1e-12


@pytest.mark.parametrize("kernel", list(KERNELS))
@pytest.mark.parametrize("bc,version", [(b, 1) for b in BCS] + [("walls_y", 2), ("walls_y", 3)])
def test_fp64_multistep_parity(cuda, kernel, bc, version):
    """20 steps: ghosts are written through by each step, walls refilled."""
    cfg = _cfg(150, 37, BCS[bc], "fp64", version=version)
    (rho, ux, uy, T), nz = _input(cfg, 20)
    p = oracle_params(cfg)
    f0 = fdlb.prepare(oeq.feq(rho, ux, uy, T) + nz, p)
    with Simulation(cfg) as sim:
        sim.set_kernel(KERNELS[kernel])
        sim.set_f(f0)
        sim.step(20)
        g = sim.get_f()
    f = fdlb.run(f0, p, 20)
    assert rel_plane_err(g, f) < 1e-11


def test_fp64_init_equilibrium_matches_oracle(cuda):
    cfg = _cfg(130, 20, BCS["periodic"], "fp64", version=3)
    rho, ux, uy, T = workloads.smooth_fields(cfg.nx, cfg.ny, 30)
    with Simulation(cfg) as sim:
        sim.init_equilibrium(rho, ux, uy, T)
        g = sim.get_f()
        r, a, b, t = sim.macros()
    f = oeq.feq(rho, ux, uy, T, 3)
    assert rel_plane_err(g, f) < 1e-14
    for x, y in ((r, rho), (a, ux), (b, uy), (t, T)):
        assert np.abs(x - y).max() < 1e-13 * max(1.0, np.abs(y).max())


_ORACLE_RUNS = {}


def _oracle_run(key, f0, p, n):
    """The oracle's n steps, shared by the kernels compared with it."""
    if key not in _ORACLE_RUNS:
        _ORACLE_RUNS[key] = fdlb.macros(fdlb.run(f0, p, n))
    return _ORACLE_RUNS[key]


@pytest.mark.parametrize("kernel", list(KERNELS))
@pytest.mark.parametrize("version", [1, 2, 3])
def test_fp32_smooth_flow_1000_steps(cuda, kernel, version):
    """FP32 storage and arithmetic (compensated temperature numerator) vs the
    FP64 oracle, on both kernels (the grid is short enough that the automatic
    choice would take the plain one) and every equilibrium version."""
    cfg = _cfg(160, 44, BCS["periodic"], "fp32", dt=1e-4, version=version)
    rho, ux, uy, T = workloads.smooth_fields(cfg.nx, cfg.ny, 40)
    p = oracle_params(cfg)
    f0 = oeq.feq(rho, ux, uy, T, version=version)
    with Simulation(cfg) as sim:
        sim.set_kernel(KERNELS[kernel])
        sim.init_equilibrium(rho, ux, uy, T)
        sim.step(1000)
        r, a, b, t = sim.macros()
    ro, ao, bo, to = _oracle_run(("smooth", version), f0, p, 1000)
    assert np.abs(r / ro - 1).max() < 1e-5
    assert np.abs(t / to - 1).max() < 1e-5
    umax = max(np.abs(ao).max(), np.abs(bo).max())
    assert np.abs(a - ao).max() < 1e-5 * umax and np.abs(b - bo).max() < 1e-5 * umax


@pytest.mark.parametrize("bc", ["walls_x", "walls_y", "reflect_y", "inflow", "diffuse_x"])
@pytest.mark.parametrize("kernel", list(KERNELS))
def test_fp32_boundaries_300_steps(cuda, bc, kernel):
    """FP32 with NEE walls (filled in FP32 each step), reflecting, inflow and
    diffuse sides vs the FP64 oracle, on both kernels."""
    cfg = _cfg(150, 37, BCS[bc], "fp32", dt=1e-4)
    rho, ux, uy, T = workloads.smooth_fields(cfg.nx, cfg.ny, 45)
    p = oracle_params(cfg)
    f0 = fdlb.prepare(oeq.feq(rho, ux, uy, T), p)
    with Simulation(cfg) as sim:
        sim.set_kernel(KERNELS[kernel])
        sim.set_f(f0.astype(np.float32))
        sim.step(300)
        r, a, b, t = sim.macros()
    ro, ao, bo, to = _oracle_run(("bc", bc), f0.astype(np.float32).astype(np.float64), p, 300)
    assert np.abs(r / ro - 1).max() < 1e-5
    assert np.abs(t / to - 1).max() < 1e-5
    umax = max(np.abs(ao).max(), np.abs(bo).max())
    assert np.abs(a - ao).max() < 1e-5 * umax and np.abs(b - bo).max() < 1e-5 * umax


@pytest.mark.parametrize("kernel", list(KERNELS))
def test_fp32_across_shocks_l1(cuda, kernel):
    """Richtmyer-Meshkov set-up (shock + interface) on 512 x 128, 200 steps,
    on both kernels."""
    cfg, (rho, ux, uy, T) = workloads.richtmyer_meshkov(nx=512, ny=128, dt=1e-5)
    p = oracle_params(cfg)
    with Simulation(cfg) as sim:
        sim.set_kernel(KERNELS[kernel])
        sim.init_equilibrium(rho, ux, uy, T)
        sim.step(200)
        r, a, b, t = sim.macros()
    ro, ao, bo, to = _oracle_run("rm", oeq.feq(rho, ux, uy, T), p, 200)
    l1 = lambda x, y: np.abs(x - y).mean() / np.abs(y).mean()
    assert l1(r, ro) < 1e-4 and l1(t, to) < 1e-4
    assert np.abs(a - ao).mean() < 1e-4 * np.abs(ao).mean()


def test_fp32_rm_crop_1000_steps(cuda):
    """The bench's shocked workload in FP32 against the oracle over 1000
    steps: a 512 x 128 crop of the Richtmyer-Meshkov 4096 x 1024 initial
    state holding the Mach-1.5 shock and the perturbed interface (x nodes
    1600-2111), with the workload's own sides, on the row-march kernel the
    bench times.  Bars: 1e-4 relative L1 across the shock and 1e-5 at every
    node (rho, T relative; u relative to max |u|)."""
    cfg, (rho, ux, uy, T) = workloads.richtmyer_meshkov()
    x0, nx, ny = 1600, 512, 128
    sl = (slice(0, ny), slice(x0, x0 + nx))
    crop = M.Config(nx=nx, ny=ny, dx=cfg.dx, dy=cfg.dy, dt=cfg.dt, s=cfg.s, bc=cfg.bc,
                    eq_version=cfg.eq_version, modified=cfg.modified, precision="fp32")
    fields = [np.ascontiguousarray(a[sl]) for a in (rho, ux, uy, T)]
    with Simulation(crop) as sim:
        sim.set_kernel(M.MRTLB_KERNEL_TILED)
        sim.init_equilibrium(*fields)
        sim.step(1000)
        r, a, b, t = sim.macros()
    ro, ao, bo, to = _oracle_run("rm_crop", oeq.feq(*fields), oracle_params(crop), 1000)
    l1 = lambda x, y: np.abs(x - y).mean() / np.abs(y).mean()
    umax = max(np.abs(ao).max(), np.abs(bo).max())
    err = {"rho": np.abs(r / ro - 1).max(), "T": np.abs(t / to - 1).max(),
           "u": max(np.abs(a - ao).max(), np.abs(b - bo).max()) / umax}
    print("RM crop FP32 vs oracle after 1000 steps: max rel rho %.2e, T %.2e, u/umax %.2e; L1 rho %.2e"
          % (err["rho"], err["T"], err["u"], l1(r, ro)))
    assert l1(r, ro) < 1e-4 and l1(t, to) < 1e-4 and np.abs(a - ao).mean() < 1e-4 * np.abs(ao).mean()
    assert max(err.values()) < 1e-5, err


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_full_size_rm_one_step_sampled(cuda, precision):
    """4096 x 1024 Richtmyer-Meshkov in the bench's launch configuration:
    one step checked at sampled nodes (tile edges, domain edges, random),
    each recomputed by the oracle from its 3 x 3 neighbourhood."""
    cfg, (rho, ux, uy, T) = workloads.richtmyer_meshkov(precision=precision)
    nz = workloads.noise((16, cfg.ny, cfg.nx), 7, 1e-4)
    p = oracle_params(cfg)
    fin = oeq.feq(rho, ux, uy, T) + nz
    if precision == "fp32":
        fin = fin.astype(np.float32)
    with Simulation(cfg) as sim:
        sim.set_f(fin)
        sim.step(1)
        out = sim.get_f()
    fin = fin.astype(np.float64)
    rng = np.random.default_rng(8)
    xs = list(rng.integers(0, cfg.nx, 1500)) + [0, 1, 2, 127, 128, 129, 2047, 2048, cfg.nx - 2, cfg.nx - 1]
    ys = list(rng.integers(0, cfg.ny, 1500)) + [0, 1, 53, 54, 55, 511, 512, 600, cfg.ny - 2, cfg.ny - 1]
    xs = np.array(xs)
    ys = np.array(ys)
    # ghost layer by the oracle's boundary rule, then 3 x 3 patches side by side
    g = fdlb._ghosts(fin, p)
    K = len(xs)
    patches = np.zeros((16, 3, 3 * K))
    for k, (x, y) in enumerate(zip(xs, ys)):
        patches[:, :, 3 * k:3 * k + 3] = g[:, y:y + 3, x:x + 3]
    pp = fdlb.Params(nx=3 * K, ny=3, dx=p.dx, dy=p.dy, dt=p.dt, s=p.s, modified=p.modified)
    ref = fdlb.step(patches, pp)[:, 1, 1::3]
    got = out[:, ys, xs].astype(np.float64)
    scale = np.abs(ref).max(axis=1, keepdims=True)
    tol = 1e-12 if precision == "fp64" else 2e-6
    assert (np.abs(got - ref) / scale).max() < tol


def test_conservation_sums(cuda):
    cfg = _cfg(257, 33, BCS["periodic"], "fp64")
    (rho, ux, uy, T), nz = _input(cfg, 50)
    f0 = oeq.feq(rho, ux, uy, T) + nz
    with Simulation(cfg) as sim:
        sim.set_f(f0)
        a = sim.reduce()
        sim.step(10)
        b = sim.reduce()
    r, jx, jy, e = oeq.conserved(f0)
    ref = np.array([r.sum(), jx.sum(), jy.sum(), e.sum()])
    assert np.allclose(a[:4], ref, rtol=1e-13, atol=1e-12 * np.abs(ref).max())
    assert np.allclose(b[:4], a[:4], rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    assert a[4] == 0.0 and b[4] > 0.0


def test_nonphysical_state_is_reported(cuda):
    cfg = _cfg(64, 8, BCS["periodic"], "fp32")
    rho, ux, uy, T = workloads.smooth_fields(cfg.nx, cfg.ny, 60)
    T[3, 5] = -0.5  # a negative temperature in the input
    with Simulation(cfg) as sim:
        sim.init_equilibrium(rho, ux, uy, T)
        sim.step(1)
        with pytest.raises(M.MrtlbError) as ei:
            sim.sync()
        assert ei.value.code == M.MRTLB_ERR_NONPHYSICAL


def test_tiled_and_plain_agree_fp32(cuda):
    cfg = _cfg(300, 70, BCS["walls_y"], "fp32")
    (rho, ux, uy, T), nz = _input(cfg, 70)
    res = []
    for k in ("plain", "tiled"):
        with Simulation(cfg) as sim:
            sim.set_kernel(KERNELS[k])
            sim.init_equilibrium(rho, ux, uy, T)
            sim.step(50)
            res.append(sim.get_f())
    # two FP32 roundings of the same arithmetic, 50 steps apart from FMA contraction
    assert rel_plane_err(res[1], res[0]) < 1e-5


def test_fp32_temperature_under_cancellation(cuda):
    """Cold, fast FP32 states (mass on one or two velocities, a thin spread)
    whose conserved moments are exact in FP32 (multiples of 2^-20 that sum
    without rounding): T = (e rho - |j|^2/2) / rho^2 from the kernels must
    match exact rational arithmetic to 1e-6.  A plain FP32 numerator loses
    up to ~6e-5 here (e rho and |j|^2/2 cancel to about 1 part in 1e4)."""
    from fractions import Fraction

    from oracle import d2v16
    V = d2v16.velocities().astype(int)
    nx, ny = 64, 16
    rng = np.random.default_rng(77)
    n = rng.integers(0, 200, (ny, nx, 16))
    for (j, i) in np.ndindex(ny, nx):
        a, b = rng.integers(0, 16, 2)
        n[j, i, a] += rng.integers(600000, 1000000)
        n[j, i, b] += rng.integers(0, 2000)
    f = np.moveaxis(n, 2, 0).astype(np.float32) * np.float32(2.0 ** -20)  # exact
    cfg = M.Config(nx=nx, ny=ny, dx=0.01, dy=0.01, dt=1e-4, s=(0,) * 4 + (1e3,) * 12,
                   bc=BCS["periodic"], precision="fp32")
    with Simulation(cfg) as sim:
        sim.set_f(f)
        T = sim.macros()[3]
    worst = 0.0
    for (j, i) in np.ndindex(ny, nx):
        fq = [Fraction(int(x), 2 ** 20) for x in n[j, i]]
        rho = sum(fq)
        jx = sum(x * int(v[0]) for x, v in zip(fq, V))
        jy = sum(x * int(v[1]) for x, v in zip(fq, V))
        e = sum(x * Fraction(int(v @ v), 2) for x, v in zip(fq, V))
        Tex = (e * rho - (jx * jx + jy * jy) / 2) / rho ** 2
        worst = max(worst, abs(T[j, i] / float(Tex) - 1))
    assert worst < 1e-6, worst


def test_fp32_conservation_drift(cuda):
    """Periodic FP32 run, 4000 steps on the tiled kernel: the sums of
    rho, j and e must not drift.  Both the Lax-Wendroff part (sum_n k_qn
    stored with an exact sum) and the collision (no conserved components)
    conserve exactly in exact arithmetic, so only unbiased rounding remains;
    a systematic error in the stored weights of 1 ulp per step would move
    the sums by ~1e-4 here."""
    cfg = _cfg(512, 128, BCS["periodic"], "fp32", dt=1e-4)
    rho, ux, uy, T = workloads.smooth_fields(cfg.nx, cfg.ny, 90)
    with Simulation(cfg) as sim:
        sim.set_kernel(M.MRTLB_KERNEL_TILED)
        sim.init_equilibrium(rho, ux, uy, T)
        a = sim.reduce()[:4]
        sim.step(4000)
        b = sim.reduce()[:4]
    scale = np.array([a[0], a[0], a[0], a[3]])  # momenta relative to mass
    assert np.all(np.abs(b - a) < 1e-6 * np.abs(scale)), (a, b)


def test_pinned_host_buffers_match_pageable(cuda):
    """set_f / get_f / macros with page-locked host buffers (read and written
    by the kernels directly) give the same bytes as with ordinary host memory
    (staged through the device)."""
    import torch
    cfg = _cfg(300, 70, BCS["outflow_x"], "fp32")
    (rho, ux, uy, T), nz = _input(cfg, 95)
    f0 = (oeq.feq(rho, ux, uy, T) + nz).astype(np.float32)
    pinned = torch.from_numpy(f0).pin_memory()
    outs = [torch.empty((cfg.ny, cfg.nx), dtype=torch.float64).pin_memory() for _ in range(4)]
    back = torch.empty_like(pinned).pin_memory()
    with Simulation(cfg) as sim:
        sim.set_f(f0)
        sim.step(3)
        want_f = sim.get_f()
        want_m = sim.macros()
        M.mrtlb_set_f(sim.ctx, pinned.data_ptr(), 0)
        sim.step(3)
        M.mrtlb_get_f(sim.ctx, back.data_ptr(), 0)
        M.mrtlb_macros(sim.ctx, *[o.data_ptr() for o in outs], 0)
    assert np.array_equal(back.numpy(), want_f)
    for o, w in zip(outs, want_m):
        assert np.array_equal(o.numpy(), w)


@pytest.mark.parametrize("kernel", list(KERNELS))
def test_fp32_uniform_state_does_not_drift(cuda, kernel):
    """A uniform FP32 state stays uniform and does not drift: every
    neighbour difference is an exact zero, so only the collision's rounding
    (of order eps^2 here) remains.  An update that rounds the same way at
    every node would move rho by ~1e-5 over these 2000 steps."""
    cfg = _cfg(256, 40, BCS["periodic"], "fp32", dt=1e-4)
    one = np.ones((cfg.ny, cfg.nx))
    with Simulation(cfg) as sim:
        sim.set_kernel(KERNELS[kernel])
        sim.init_equilibrium(one, 0.1 * one, -0.05 * one, one)
        r0, a0, b0, t0 = sim.macros()
        sim.step(2000)
        r, a, b, t = sim.macros()
    assert np.abs(r / r0 - 1).max() < 1e-6 and np.abs(t / t0 - 1).max() < 1e-6
    assert np.abs(a - a0).max() < 1e-6 and np.abs(b - b0).max() < 1e-6


def test_bounded_wait_reports_a_timeout_and_the_context_recovers(cuda):
    """A kernel wait that cannot complete gives up after its bound (about
    2 s): the host reads MRTLB_ERR_TIMEOUT, the error word is cleared, and
    the context keeps stepping correctly."""
    import time
    cfg = _cfg(64, 8, BCS["periodic"], "fp64")
    (rho, ux, uy, T), nz = _input(cfg, 97)
    p = oracle_params(cfg)
    f0 = fdlb.prepare(oeq.feq(rho, ux, uy, T) + nz, p)
    with Simulation(cfg) as sim:
        sim.set_f(f0)
        t0 = time.perf_counter()
        rc = M.mrtlb_selftest_wait(sim.ctx)
        waited = time.perf_counter() - t0
        assert rc == M.MRTLB_ERR_TIMEOUT
        assert 1.5 < waited < 30.0
        sim.step(3)
        sim.sync()
        g = sim.get_f()
    assert rel_plane_err(g, fdlb.run(f0, p, 3)) < 1e-12
