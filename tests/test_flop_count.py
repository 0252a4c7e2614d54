"""The flops of one node update, counted by running the step kernels' own
per-node templates on the host with an operation-counting number type
(tests/flopcount/step_flops.cu), against a closed form for the advection
and the constants bench.py reports."""
import json
import os
import shutil
import subprocess

import pytest

import bench

HERE = os.path.dirname(os.path.abspath(__file__))


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


@pytest.fixture(scope="module")
def counts(tmp_path_factory):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("flops") / "step_flops")
    src = os.path.join(HERE, "flopcount", "step_flops.cu")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-O1",
                    "-diag-suppress", "177,20011,20014", "-o", exe, src], check=True, capture_output=True)
    return json.loads(subprocess.run([exe], check=True, capture_output=True, text=True).stdout)


def test_advection_count_matches_the_closed_form(counts):
    # per velocity: f - C, then (f_n - f) k + v for each of its two (axis
    # shells: one) moving directions' two neighbours: 8 axis velocities of
    # 1 + 2*3 flops and 8 diagonal ones of 1 + 4*3
    for prec in ("fp32", "fp64"):
        assert counts[prec]["advect"] == 8 * 7 + 8 * 13
        assert counts[prec]["finite"] == 1


def test_precisions_differ_only_in_the_macroscopic_state(counts):
    assert counts["fp32"]["collide"] == counts["fp64"]["collide"]
    # FP32: compensated numerator and a Newton-refined reciprocal; FP64: the
    # plain numerator and one division
    assert counts["fp32"]["arrive"] > counts["fp64"]["arrive"]
    assert counts["fp64"]["divs"] == 1 and counts["fp32"]["sfu"] == 1


def test_bench_reports_the_counted_flops(counts):
    assert bench.STEP_FLOPS_PER_LUP == {p: counts[p]["total"] for p in ("fp32", "fp64")}
