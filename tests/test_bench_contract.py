"""The benchmark's reference arm on the CPU: `bench.py --impl reference`
times the FP64 oracle on the host cores and prints one JSON line with the
GPU arm's metric, unit and workload name; under a multi-rank launch only
rank 0 prints.  CPU only (the oracle needs no GPU)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None):
    env = dict(os.environ)
    for k in ("RANK", "LOCAL_RANK", "WORLD_SIZE"):
        env.pop(k, None)
    env.update(extra_env or {})
    return subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


@pytest.fixture(scope="module")
def line():
    p = _run()
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [s for s in p.stdout.splitlines() if s.startswith("{")]
    assert len(lines) == 1, p.stdout
    return json.loads(lines[0])


def test_reference_line_keeps_the_contract(line):
    sys.path.insert(0, ROOT)
    import bench

    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["higher_is_better"] is True and line["scaling"] == "weak"
    assert line["steps"] == 1 and line["warmup"] == 3 and line["n_gpus"] == 1
    assert line["value"] > 0.0 and line["ms_per_step"] > 0.0
    assert line["vs_baseline"] is None and line["data"] == "synthetic" and line["dtype"] == "f64"
    # the GPU arm's workload (512^3, 2,880 spheres, 6 levels), the sample beside it
    assert line["config"]["workload"] == bench.workload_name(512, 2880, 6, 4e-6)
    assert line["config"]["cells"] == 512 ** 3
    assert "128^3" in line["config"]["sample"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1 and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_prints_on_rank_zero_only():
    p = _run({"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"})
    assert p.returncode == 0, p.stderr[-2000:]
    assert not [s for s in p.stdout.splitlines() if s.startswith("{")]
