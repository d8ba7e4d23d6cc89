"""bench.py's reference arm (the FP64 oracle on host cores) keeps its JSON
contract: one line on rank 0 with the metric, a positive value, the oracle
described as the CPU baseline and an end-to-end entry with no copies; other
ranks print nothing and exit 0."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env):
    env = dict(os.environ)
    env.update(extra_env)
    env["CUDA_VISIBLE_DEVICES"] = ""
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1", "--warmup", "0"]
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    p = _run({"RANK": "0", "WORLD_SIZE": "1"})
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "dtype", "data", "config"):
        assert key in d, key
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "workload" in d["config"]


def test_reference_arm_other_ranks_do_no_work():
    p = _run({"RANK": "1", "WORLD_SIZE": "2"})
    assert p.returncode == 0, p.stderr[-2000:]
    assert p.stdout.strip() == ""


def test_many_slice_workloads_time_the_oracle_on_one_problem():
    """The CPU baseline of the batched, ragged and differentiable workloads:
    the oracle in a single-threaded child on one problem's first update; for
    the ragged workload that problem is its first draw."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_1705_07497_gb300 import inputs

    wl = inputs.WORKLOADS["ragged_64"]
    one = bench.single_problem(wl)
    n, a, d, nb, seed = inputs.ragged_problems(wl)[0]
    assert (one["n"], one["n_angles_total"], one["keep_every"], one["n_bins"], one["seed"]) == (n, a, d, nb, seed)
    assert bench.single_problem(inputs.WORKLOADS["grad_256x16"]) is inputs.WORKLOADS["grad_256x16"]
    cb = bench.oracle_slice_baseline("grad_256x16", 3000, 3100, " (note)")
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["unit"] == "slices/s"
    assert cb["value"] > 0 and cb["sample"].endswith("(note)")
