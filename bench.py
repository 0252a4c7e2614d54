#!/usr/bin/env python
"""Throughput of the MRT FD-LB step (arXiv:1106.0785) on GB300.

Default workload: Richtmyer-Meshkov, 4096 x 1024 nodes, FP32 distributions
with a compensated temperature numerator (a Mach-1.5 shock onto a cosine-perturbed
light/heavy interface; seeded synthetic fields).  One bench step = one time
step of the whole path: one fused step kernel (macroscopic recovery,
velocity gradients, moments, equilibria, modified collision, Lax-Wendroff
advection, forward-Euler update) that also writes the boundary ghost layer
of the new state (outflow in x, periodic in y).

Printed JSON line (rank 0):
  value      MLUPS (million lattice-node updates / s), whole job, inputs
             resident in HBM, CUDA events on the library's stream
  e2e        the same through the C ABI with host buffers: every step copies
             f in from pinned host memory and rho, u, T back
  roofline   step kernel: algorithmic 128 B / node update (16 FP32 reads +
             16 writes) / its mean launch time (the timed region's time over
             its launches, the step kernel being its only kernel), against
             measured HBM copy bandwidth
  fp64_mlups the all-FP64 path on the same input
  batched    64 seeded uneven instances in one persistent launch per step:
             MLUPS, fraction of the copy bandwidth at 128 B / node update,
             and the kernel's DRAM bytes per launch from its ncu summary
             (traffic, null once the kernel's sources changed)
  fwd_adj    K = 64 forward + adjoint steps with sqrt(K) checkpoints, and
             with every state stored, against 320 B / node update
  compute    the step's flop rate (counted flops per node update) against
             fused multiply-add ceilings measured on the device
  small      microseconds per step of the latency-bound small configurations
             (Sod 400 x 4 FP64, Couette 4 x 200 FP64 and FP32)
  cpu_baseline  the FP64 oracle (its plain-C step) on a crop of the same input,
                one single-threaded process per host core (and one alone:
                single_core_mlups)
  oracle_parity the FP32 CUDA path on that crop after the same steps, against
                the oracle's result (largest errors in rho, u, T)

Multi-GPU (torchrun): every rank advances its own replica (weak scaling, no
data-path collective); the max time over ranks is reported.
"""
import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NX, NY = 4096, 1024
BYTES_PER_LUP_FP32 = 128
# Floating-point operations of one node update (a fused multiply-add counts
# two), counted by running the step kernels' own per-node templates with an
# operation-counting number type (tests/flopcount/step_flops.cu; the CPU
# test suite keeps these equal to its output).
STEP_FLOPS_PER_LUP = {"fp32": 539, "fp64": 521}
CROP = (1600, 0, 512, 128)      # x0, y0, nx, ny of the CPU-baseline crop
REF_CROP = (1900, 0, 128, 64)   # per-step sample of the reference arm
PARITY_STEPS = 1000             # the CUDA path against the oracle on CROP after at least this many steps


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--fp64-steps", type=int, default=30)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-steps", type=int, default=500)
    ap.add_argument("--adjoint-steps", type=int, default=64)
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--cpu-cores", type=int, default=0, help="oracle processes (0: one per host core)")
    ap.add_argument("--ref-cores", type=int, default=0, help="reference-arm processes (0: one per host core)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed helpers (one process per GPU; replicas)
# ---------------------------------------------------------------------------
def dist_init(backend):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device=None):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,"
             "clocks.mem,clocks.max.mem")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons, mem, mmax = [], None, set(), [], None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            try:
                mem.append(float(parts[9]))
                mmax = float(parts[10])
            except (ValueError, IndexError):
                pass
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        sm.sort()
        mem.sort()
        out = {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": smax, "reasons": sorted(reasons),
               "samples": len(sm)}
        if mem:
            out.update(mem_mhz=mem[len(mem) // 2], mem_max_mhz=mmax)
        return out


# ---------------------------------------------------------------------------
# roofline inputs
# ---------------------------------------------------------------------------
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


STEP_SOURCES = ("step_tiled.cu", "march.cuh", "march_pair.cuh", "pair.cuh", "physics.cuh", "kernels.cuh")
BATCH_SOURCES = ("batch.cu", "march.cuh", "march_pair.cuh", "pair.cuh", "physics.cuh", "kernels.cuh")


def kernel_source_hash(names=STEP_SOURCES):
    """Hash of a kernel's sources without // comments and blank lines, so
    that only changes of the code itself invalidate a profile."""
    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, "paper_1106_0785_gb300", "csrc", name)) as fh:
            for line in fh:
                code = re.sub(r"//.*", "", line).strip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def profiled_traffic(profile="step_pair_fp32_rm4096x1024.md", names=STEP_SOURCES):
    """DRAM bytes per launch of a kernel from its committed ncu summary, if
    it was taken on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", profile)
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    s = re.search(r"kernel_source_sha:\s*([0-9a-f]+)", text)
    if not m or not s or s.group(1) != kernel_source_hash(names):
        return None
    return float(m.group(1))


# ---------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on a crop of the same input
# ---------------------------------------------------------------------------
def _crop_problem(crop):
    import numpy as np

    from oracle import equilibrium as oeq
    from oracle import fdlb
    from paper_1106_0785_gb300 import workloads

    cfg, (rho, ux, uy, T) = workloads.richtmyer_meshkov(nx=NX, ny=NY)
    x0, y0, nx, ny = crop
    sl = (slice(y0, y0 + ny), slice(x0, x0 + nx))
    p = fdlb.Params(nx=nx, ny=ny, dx=cfg.dx, dy=cfg.dy, dt=cfg.dt, s=np.asarray(cfg.s),
                    sides=tuple(fdlb.Side(side[0], *side[1:]) for side in cfg.bc))
    return p, oeq.feq(rho[sl], ux[sl], uy[sl], T[sl])


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), or None."""
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
        for line in r.stdout.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def host_cores():
    """Cores this process may run on (the affinity mask, else the count)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _until(t_start):
    while True:
        d = t_start - time.time()
        if d <= 0:
            return
        time.sleep(min(d, 0.05))


def cpu_baseline_worker(seconds, out=None, t_start=0.0, min_steps=0):
    """One thread: the oracle's C step on the crop for about `seconds`, from
    t_start (wall clock) so that the workers of one measurement run
    together.  With `out`, the run then goes on (untimed) to at least
    min_steps steps and saves the first and last states for the parity
    check."""
    import numpy as np

    from oracle import cfdlb
    p, f0 = _crop_problem(CROP)
    r = cfdlb.Runner(f0, p)
    r.run(1)  # warm-up (counted: the result is compared step for step)
    _until(t_start)
    n, t0 = 1, time.perf_counter()
    while True:
        r.run(1)
        n += 1
        el = time.perf_counter() - t0
        if (el >= seconds and n >= 3) or n >= 100000:
            break
    timed = n - 1
    if out:
        if n < min_steps:
            r.run(min_steps - n)
            n = min_steps
        np.savez(out, f0=f0, fn=r.f)
    print(json.dumps({"steps": n, "timed_steps": timed, "seconds": el, "nodes": p.nx * p.ny}))


def _run_workers(codes, timeout):
    """Run one single-threaded Python worker per code string at once (fresh
    processes: no state of this process, GPU or otherwise, is inherited);
    returns their last stdout lines parsed as JSON, or raises."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    procs = [subprocess.Popen([sys.executable, "-c", c], cwd=ROOT, env=env, stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True) for c in codes]
    outs = []
    try:
        for pr in procs:
            so, se = pr.communicate(timeout=timeout)
            if pr.returncode != 0:
                raise RuntimeError(se[-300:])
            outs.append(json.loads(so.strip().splitlines()[-1]))
    finally:
        for pr in procs:  # after a failure, stop the workers still running
            if pr.poll() is None:
                pr.kill()
                pr.wait()
    return outs


def cpu_baseline(seconds, dev=None, cores=None):
    """The oracle's rate on the crop on every host core: one independent
    single-threaded process per core, started together; and, when a device
    is given, the CUDA path's error against the oracle's result on that crop
    after the same number of steps (FP32, the bench's precision): returns
    (cpu_baseline, oracle_parity)."""
    import tempfile

    from oracle import cfdlb
    cfdlb.build()  # once, before the workers start
    n = cores or host_cores()
    with tempfile.TemporaryDirectory() as tmp:
        out = os.path.join(tmp, "oracle_crop.npz")
        t_start = time.time() + 3.0 + 0.1 * n  # after every worker has imported and warmed up
        keep = dev is not None  # the first worker also serves the parity check
        codes = ["import bench; bench.cpu_baseline_worker(%r, %r, %r, %d)"
                 % (seconds, out if (i == 0 and keep) else None, t_start, PARITY_STEPS if (i == 0 and keep) else 0)
                 for i in range(n)]
        try:
            ds = _run_workers(codes, timeout=600 + 10 * n)
        except (RuntimeError, subprocess.SubprocessError) as e:
            return {"error": str(e)[-300:]}, None
        parity = crop_parity(out, ds[0]["steps"], dev) if dev is not None else None
    per = [d["nodes"] * d["timed_steps"] / d["seconds"] / 1e6 for d in ds]
    # the same step on one core with the others idle (the single-thread rate)
    single_s = max(1.0, seconds / 5.0)
    try:
        d1 = _run_workers(["import bench; bench.cpu_baseline_worker(%r, None, %r, 0)"
                           % (single_s, time.time() + 3.0)], timeout=300)[0]
        single = d1["nodes"] * d1["timed_steps"] / d1["seconds"] / 1e6
    except (RuntimeError, subprocess.SubprocessError):
        single = None
    x0, y0, nx, ny = CROP
    base = {"value": sum(per), "unit": "MLUPS", "cores": n, "kind": "oracle",
            "per_core_mlups": sum(per) / n, "single_core_mlups": single, "cpu_model": cpu_model(),
            "sample": "FP64 oracle (its plain-C step), %d single-threaded processes at once (one per host core), each "
                      "%d-%d timed steps of a %dx%d crop (x %d-%d, y %d-%d) of the Richtmyer-Meshkov 4096x1024 "
                      "initial state for about %.0f s; value = the sum of their rates; single_core_mlups: one "
                      "such process alone for about %.0f s"
                      % (n, min(d["timed_steps"] for d in ds), max(d["timed_steps"] for d in ds), nx, ny,
                         x0, x0 + nx - 1, y0, y0 + ny - 1, seconds, single_s)}
    return base, parity


def crop_parity(path, steps, dev):
    """The FP32 CUDA path (the row-march kernel the bench times) on the
    oracle's crop problem (the workload's sides: the post-shock inflow on
    the left, outflow on the right, periodic in y), from the same
    initial state for the same steps: the largest relative error in rho and
    T and in u relative to max |u|."""
    import numpy as np

    from oracle import fdlb
    from paper_1106_0785_gb300 import mrtlb as M
    from paper_1106_0785_gb300 import workloads
    from paper_1106_0785_gb300.simulation import Simulation

    z = np.load(path)
    cfg, _ = workloads.richtmyer_meshkov(nx=NX, ny=NY)
    x0, y0, nx, ny = CROP
    crop = M.Config(nx=nx, ny=ny, dx=cfg.dx, dy=cfg.dy, dt=cfg.dt, s=cfg.s, bc=cfg.bc,
                    eq_version=cfg.eq_version, modified=cfg.modified, precision="fp32")
    with Simulation(crop, device=dev) as sim:
        sim.set_kernel(M.MRTLB_KERNEL_TILED)  # the kernel the bench times (the crop is short enough
        sim.set_f(z["f0"].astype(np.float32))  # that the automatic choice would take the plain one)
        sim.step(steps)
        r, ux, uy, T = sim.macros()
    r0, ux0, uy0, T0 = fdlb.macros(z["fn"])
    umax = max(np.abs(ux0).max(), np.abs(uy0).max())
    return {"steps": int(steps), "precision": "fp32", "against": "the FP64 oracle",
            "sample": "the cpu_baseline crop",
            "max_rel_err_rho": float((np.abs(r - r0) / np.abs(r0)).max()),
            "max_err_u_over_umax": float(max(np.abs(ux - ux0).max(), np.abs(uy - uy0).max()) / umax),
            "max_rel_err_T": float((np.abs(T - T0) / np.abs(T0)).max())}


# ---------------------------------------------------------------------------
# reference arm: the oracle as it stands on the host cores
# ---------------------------------------------------------------------------
def reference_worker(warmup, steps, t_start):
    """One thread: `warmup` then `steps` steps of the oracle's C step on the
    reference crop, the timed steps from t_start (wall clock)."""
    from oracle import cfdlb
    p, f = _crop_problem(REF_CROP)
    r = cfdlb.Runner(f, p)
    for _ in range(warmup):
        r.run(1)
    _until(t_start)
    t0 = time.perf_counter()
    for _ in range(steps):
        r.run(1)
    print(json.dumps({"seconds": time.perf_counter() - t0, "nodes": p.nx * p.ny}))


def run_reference(args, world, rank):
    """The oracle as it stands on every host core: one single-threaded
    process per core, each advancing its own copy of the crop, timed
    together; a bench step is one time step of every copy."""
    if rank != 0:
        return
    from oracle import cfdlb
    cfdlb.build()  # once, before the workers start
    n = args.ref_cores or host_cores()
    t_start = time.time() + 3.0 + 0.1 * n + 0.05 * args.warmup
    ds = _run_workers(["import bench; bench.reference_worker(%d, %d, %r)" % (args.warmup, args.steps, t_start)
                       for _ in range(n)], timeout=600 + 10 * n)
    el = max(d["seconds"] for d in ds)
    nodes = ds[0]["nodes"]
    mlups = n * nodes * args.steps / el / 1e6
    x0, y0, nx, ny = REF_CROP
    sample = ("FP64 oracle (its plain-C step), %d single-threaded processes at once (one per host core), each one time "
              "step of its own %dx%d crop (x %d-%d, y %d-%d) of the Richtmyer-Meshkov 4096x1024 initial "
              "state per bench step" % (n, nx, ny, x0, x0 + nx - 1, y0, y0 + ny - 1))
    line = {
        "impl": "reference", "metric": "MLUPS, FP32 forward step (Richtmyer-Meshkov 4096x1024)",
        "value": mlups, "unit": "MLUPS", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "richtmyer_meshkov_4096x1024", "nx": NX, "ny": NY,
                   "precision": "fp64 (the oracle)", "parallelism": "host cores, %d processes" % n,
                   "sample": sample},
        "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": n, "kind": "oracle", "sample": sample,
                         "cpu_model": cpu_model()},
        "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------
def run_mine(args, world, rank, local):
    import numpy as np
    import torch

    import __graft_entry__
    from paper_1106_0785_gb300 import mrtlb as M
    from paper_1106_0785_gb300 import workloads
    from paper_1106_0785_gb300.simulation import Simulation

    __graft_entry__.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfg, fields = workloads.richtmyer_meshkov(nx=NX, ny=NY, precision="fp32")
    nodes = NX * NY
    sim = Simulation(cfg, device=dev)
    sim.init_equilibrium(*fields)
    stream = sim.stream
    sim.step(args.warmup)
    sim.sync()

    # ---- timed region: K steps through mrtlb_step (the library's time loop,
    # CUDA graphs), inputs resident in HBM ---------------------------------
    clk = ClockSampler(local)
    clk.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier(world)
    ms = e0.elapsed_time(e1)
    clocks = clk.stop()
    sim.sync()  # surfaces any non-physical state met during the run
    ms_max = max_over_ranks(ms, world, dev)
    value = world * nodes * args.steps / (ms_max / 1e3) / 1e6
    launches = M.mrtlb_launches_per_step(sim.ctx) * args.steps

    # ---- roofline of the step kernel --------------------------------------
    # The step kernel is the only kernel of the timed region (one launch per
    # step), so its mean launch duration is at most the region's event time
    # over its launches (the gaps between launches included).  For reference,
    # the same kernel timed with events around each launch (which replaces
    # the graphs by single launches and adds the events' own overhead).
    peak, peak_src = measured_peaks()
    kavg_s = ms_max / 1e3 / max(launches, 1)
    achieved = BYTES_PER_LUP_FP32 * nodes / kavg_s / 1e9
    nref = min(args.steps, 500)
    M.mrtlb_timing_begin(sim.ctx, nref)
    sim.step(nref)
    kms, nlaunch = M.mrtlb_timing_end(sim.ctx)
    traffic = profiled_traffic()
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                "kernel": "step_pair_kernel<128,4,4>", "kernel_ms_mean": kavg_s * 1e3,
                "kernel_ms_source": "timed region / launches (an upper bound: gaps included)",
                "kernel_ms_events": kms / max(nlaunch, 1),
                "peak_source": peak_src + " (MEASURED_PEAKS.json hbm_gbs, copy)"}

    # ---- compute side: measured FMA ceilings, outside the timed region -----
    ceil = {k: M.mrtlb_measure_peak(v) for k, v in (("fp32", M.MRTLB_PEAK_FP32),
                                                    ("fp32_pair", M.MRTLB_PEAK_FP32_PAIR),
                                                    ("fp64", M.MRTLB_PEAK_FP64))}
    step_tflops = STEP_FLOPS_PER_LUP["fp32"] * nodes / kavg_s / 1e12
    compute = {"unit": "TFLOP/s", "flops_per_lup": STEP_FLOPS_PER_LUP,
               "step_fp32": step_tflops, "ceiling_fp32": ceil["fp32"],
               "ceiling_fp32_pair": ceil["fp32_pair"], "ceiling_fp64": ceil["fp64"],
               "step_frac_of_fp32": step_tflops / ceil["fp32"] if ceil["fp32"] > 0 else None}

    # ---- e2e through the C ABI with host buffers ---------------------------
    f_host = torch.empty((16, NY, NX), dtype=torch.float32, pin_memory=True)
    sim.get_f()  # warm the staging buffer
    M.mrtlb_get_f(sim.ctx, f_host.data_ptr(), 0)
    outs = [torch.empty((NY, NX), dtype=torch.float64, pin_memory=True) for _ in range(4)]
    ke = max(1, args.e2e_steps)
    for _ in range(2):
        M.mrtlb_set_f(sim.ctx, f_host.data_ptr(), 0)
        M.mrtlb_step(sim.ctx, 1)
        M.mrtlb_macros(sim.ctx, *[o.data_ptr() for o in outs], 0)
    barrier(world)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(ke):
        M.mrtlb_set_f(sim.ctx, f_host.data_ptr(), 0)      # H2D of f^n (pinned)
        M.mrtlb_step(sim.ctx, 1)
        M.mrtlb_macros(sim.ctx, *[o.data_ptr() for o in outs], 0)  # D2H of rho, u, T
    torch.cuda.synchronize(dev)
    el = max_over_ranks(time.perf_counter() - t0, world, dev)
    e2e = {"value": world * nodes * ke / el / 1e6, "unit": "MLUPS",
           "h2d_bytes_per_step": int(f_host.numel() * 4),
           "d2h_bytes_per_step": int(sum(o.numel() for o in outs) * 8)}
    sim.close()

    # ---- forward + adjoint (stored states) on the same input ------------------
    fwd_adj = None
    if not args.no_adjoint:
        fwd_adj = run_fwd_adj(args, world, dev, cfg, fields, nodes)

    # ---- the all-FP64 path on the same input --------------------------------
    cfg64, _ = workloads.richtmyer_meshkov(nx=NX, ny=NY, precision="fp64")
    sim64 = Simulation(cfg64, device=dev)
    sim64.init_equilibrium(*fields)
    sim64.step(3)
    sim64.sync()
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    a0.record(sim64.stream)
    sim64.step(args.fp64_steps)
    a1.record(sim64.stream)
    torch.cuda.synchronize(dev)
    ms64 = max_over_ranks(a0.elapsed_time(a1), world, dev)
    sim64.sync()
    sim64.close()
    fp64_mlups = world * nodes * args.fp64_steps / (ms64 / 1e3) / 1e6
    compute["step_fp64"] = STEP_FLOPS_PER_LUP["fp64"] * fp64_mlups / world / 1e6
    compute["step_frac_of_fp64"] = compute["step_fp64"] / ceil["fp64"] if ceil["fp64"] > 0 else None

    # ---- the batched set: 64 uneven Sod-type / Couette instances -----------
    batched = None
    if not args.no_batch:
        batched = run_batched(args, world, dev)

    # ---- the small, latency-bound configurations ----------------------------
    small = run_small(dev)

    if rank != 0:
        return
    line = {
        "metric": "MLUPS, FP32 forward step (Richtmyer-Meshkov 4096x1024)",
        "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "richtmyer_meshkov_4096x1024", "nx": NX, "ny": NY,
                   "precision": "fp32 storage and arithmetic, compensated temperature numerator",
                   "l2": "inputs larger than L2 (268 MB per f copy)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "e2e": e2e,
        "gpu_launches": launches,
        "roofline": roofline,
        "compute": compute,
        "fp64_mlups": fp64_mlups,
        "fp64_ms_per_step": ms64 / args.fp64_steps,
        "batched": batched,
        "fwd_adj": fwd_adj,
        "small": small,
        "clocks": clocks,
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"], line["oracle_parity"] = cpu_baseline(args.cpu_seconds, dev, args.cpu_cores or None)
    print(json.dumps(line), flush=True)


def run_fwd_adj(args, world, dev, cfg, fields, nodes):
    """K FP32 steps forward, then the adjoint back to the initial state
    (seed: dL/dT = 1 on every node), two ways: with sqrt(K) checkpointing
    (segments of ceil(sqrt(K)) steps; every segment but the last is
    recomputed from its checkpoint in the backward pass) and with every
    state stored (no recomputation).  MLUPS = nodes * K / total time;
    algorithmic bytes 320 / node update (forward 128 + adjoint: read f, read
    lambda, write lambda, 64 each); the recomputed steps' traffic is extra,
    not counted.  Each timed pass follows a warm-up pass of the same shape,
    so it reuses the library's buffers and plans, as every pass of a
    gradient loop after the first does."""
    import torch

    from paper_1106_0785_gb300.simulation import Simulation

    K = args.adjoint_steps
    peak, _ = measured_peaks()
    seed = torch.zeros((4, cfg.ny, cfg.nx), dtype=torch.float64, device=dev)
    seed[3] = 1.0

    def one(interval):
        sim = Simulation(cfg, device=dev)
        seg = max(1, min(interval, K))
        nseg = (K + seg - 1) // seg
        sim.init_equilibrium(*fields)
        sim.adjoint_forward(K, interval=seg)  # warm-up (allocations, graphs)
        sim.adjoint_backward(dL_dmacros=seed, want_df0=False)
        sim.init_equilibrium(*fields)
        barrier(world)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        sim.adjoint_forward(K, interval=seg)
        ds, _ = sim.adjoint_backward(dL_dmacros=seed, want_df0=False)
        torch.cuda.synchronize(dev)
        el = max_over_ranks(time.perf_counter() - t0, world, dev)
        sim.close()
        gbs = 320 * nodes * K / el / 1e9
        recomputed = (nseg - 1) * seg if nseg > 1 else 0
        held = seg + (nseg if nseg > 1 else 0) + 2  # segment slots, checkpoints, two adjoint buffers
        return {"segment_steps": seg, "segments": nseg, "recomputed_steps": recomputed,
                "mlups": world * nodes * K / el / 1e6, "seconds": el,
                "algorithmic_gbs": gbs, "frac_of_hbm": gbs / peak,
                "state_memory_bytes": held * sim.state_bytes,
                "recompute_bytes": recomputed * BYTES_PER_LUP_FP32 * nodes,
                "dL_ds_visc": float(ds[4] + ds[5]), "dL_ds_cond": float(ds[6] + ds[7])}

    ck = one(int(math.ceil(math.sqrt(K))))
    stored = one(K)
    out = {"K": K, "checkpointing": "sqrt(K)"}
    out.update(ck)
    out["stored_states"] = stored
    return out


def run_small(dev):
    """Microseconds per step of the two small configurations, which launch
    latency rather than HBM bounds: the Sod tube (400 x 4, FP64, its 1500
    steps to t = 0.015) and thermal Couette flow (4 x 200, FP64 and FP32,
    2000 steps), each as the library's graph-replayed time loop after a
    warm-up."""
    import torch

    from paper_1106_0785_gb300 import workloads
    from paper_1106_0785_gb300.simulation import Simulation

    out = {}
    for name, (cfg, fields), steps in (
            ("sod_400x4_fp64", workloads.sod(precision="fp64"), 1500),
            ("couette_4x200_fp64", workloads.couette(Pr=2.0, precision="fp64"), 2000),
            ("couette_4x200_fp32", workloads.couette(Pr=2.0, precision="fp32"), 2000)):
        with Simulation(cfg, device=dev) as sim:
            sim.init_equilibrium(*fields)
            sim.step(128)
            sim.sync()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(sim.stream)
            sim.step(steps)
            e1.record(sim.stream)
            torch.cuda.synchronize(dev)
            sim.sync()
            out[name + "_us_per_step"] = 1e3 * e0.elapsed_time(e1) / steps
    return out


def run_batched(args, world, dev):
    """64 seeded instances (grids 128-2048 x 4-256, Sod-type and Couette,
    Pr 0.3-3) in one persistent launch per step, time loop as CUDA graphs,
    tile shape from the autotuner (cached outside the repository)."""
    import tempfile

    import torch

    from paper_1106_0785_gb300 import workloads
    from paper_1106_0785_gb300.simulation import Batch, Simulation

    insts = workloads.batched_instances(64, precision="fp32")
    sims = []
    for cfg, fields in insts:
        s = Simulation(cfg, device=dev)
        s.init_equilibrium(*fields)
        sims.append(s)
    b = Batch(sims)
    cache = os.path.join(tempfile.gettempdir(), "mrtlb_batch_tune.txt")
    b.tune(cache, trial_steps=10)
    b.step(64)
    b.sync()
    stream = sims[0].stream
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    b.step(args.batch_steps)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier(world)
    b.sync()
    ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
    nodes = b.nodes
    bx, seglen, ntiles, grid = b.tiles
    peak, _ = measured_peaks()
    per_step_s = ms / 1e3 / args.batch_steps
    gbs = BYTES_PER_LUP_FP32 * nodes / per_step_s / 1e9
    out = {"instances": len(insts), "nodes": nodes, "steps": args.batch_steps,
           "mlups": world * nodes * args.batch_steps / (ms / 1e3) / 1e6,
           "ms_per_step": ms / args.batch_steps,
           "step_gbs": gbs, "step_frac_of_hbm": gbs / peak,
           "tiles": {"bx": bx, "seglen": seglen, "ntiles": ntiles, "grid": grid},
           "launches_per_step": 2, "graph_steps": 64}
    # DRAM bytes of one launch of the batched kernel (ncu, its committed
    # summary, while the kernel's sources hash the same), against the
    # algorithmic 128 B per node update
    traffic = profiled_traffic("step_batched_pair_fp32_64instances.md", BATCH_SOURCES)
    out["traffic"] = traffic
    out["traffic_over_algorithmic"] = traffic / (BYTES_PER_LUP_FP32 * nodes) if traffic else None
    b.close()
    for s in sims:
        s.close()
    return out


def main():
    args = parse()
    if args.impl == "reference":
        world, rank, _ = dist_init("gloo")
        run_reference(args, world, rank)
        return
    world, rank, local = dist_init("nccl")
    run_mine(args, world, rank, local)


if __name__ == "__main__":
    main()
