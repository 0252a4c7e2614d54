"""The bench's multi-rank logic on CPU (gloo, world size 2): replicas with
a barrier and a max over ranks, and the reference arm under torchrun
(rank 0 alone runs and prints one line; the other rank exits cleanly)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    w, r, _ = bench.dist_init("gloo")
    bench.barrier(w)
    # each rank "timed" a different duration: the job takes the slowest
    slowest = bench.max_over_ranks(1.0 + r, w)
    import torch.distributed as dist
    dist.destroy_process_group()
    with open(os.path.join(out, "rank%d.json" % rank), "w") as fh:
        json.dump({"world": w, "rank": r, "slowest": slowest}, fh)


def test_max_over_ranks_and_barrier_gloo(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    got = [json.load(open(tmp_path / ("rank%d.json" % r))) for r in range(2)]
    assert [g["rank"] for g in got] == [0, 1]
    assert all(g["world"] == 2 and g["slowest"] == 2.0 for g in got)


@pytest.mark.slow
def test_reference_arm_under_torchrun_two_ranks():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["cpu_baseline"]["cores"] >= 1


def test_cpu_baseline_runs_one_oracle_process_per_core():
    """The oracle baseline: independent single-threaded processes started
    together; the value is the sum of their rates, the core count is the
    number of processes."""
    sys.path.insert(0, ROOT)
    import bench
    base, parity = bench.cpu_baseline(0.5, None, 2)
    assert parity is None and "error" not in base, base
    assert base["cores"] == 2 and base["kind"] == "oracle" and base["value"] > 0
    assert abs(base["per_core_mlups"] * 2 - base["value"]) < 1e-9 * base["value"]
    assert "2 single-threaded processes" in base["sample"]
    # and one such process alone (the single-thread rate)
    assert base["single_core_mlups"] > 0
