"""CPU checks of bench.py's reference arm (the FP64 oracle timed on the host cores):
one JSON line with the keys of the benchmark contract; ranks other than 0 do no work
and print nothing."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    r = _run({})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 0 and d["higher_is_better"] is True
    assert d["config"]["workload"].startswith("lid-driven cavity 256x256")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_quietly():
    r = _run({"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def test_gpu_arm_fails_loudly_without_a_gpu():
    """No CPU fallback: without CUDA the GPU arm exits non-zero and prints no result."""
    import pytest
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    r = subprocess.run([sys.executable, "bench.py", "--steps", "1", "--warmup", "0", "--no-cpu-baseline"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0
    assert not any(ln.lstrip().startswith("{") for ln in r.stdout.splitlines())


def test_stopping_rule_of_the_batched_solves():
    """The retirement rule of `--workload batch-solve` (Sec. IV residual checked every
    interval): converged below the target; diverged on a NaN residual; stalled when
    `stall` checks in a row bring no minimum 1 % below the last one; capped at the step
    cap.  An infinite residual (no snapshot motion yet) is none of these."""
    sys.path.insert(0, ROOT)
    import bench
    r = bench.Retire(target=1e-6, cap=10_000, stall=3)
    assert r(float("inf"), 1000) is None
    assert r(1e-3, 2000) is None
    assert r(0.995e-3, 3000) is None              # less than 1 % lower: no new minimum
    assert r(0.994e-3, 4000) is None
    assert r(0.5e-3, 5000) is None                # a new minimum resets the count
    assert r(0.5e-3, 6000) is None
    assert r(0.5e-3, 7000) is None
    assert r(0.5e-3, 8000) == "stalled"
    assert bench.Retire(1e-6, 10_000, 3)(0.9e-6, 1000) == "converged"
    assert bench.Retire(1e-6, 10_000, 3)(float("nan"), 1000) == "diverged"
    assert bench.Retire(1e-6, 2000, 50)(1e-3, 2000) == "capped"
