"""The benchmark's command-line contract, checked without a GPU: the oracle
(reference) arm prints one JSON line with every required key, on the metric
and unit of the GPU arm; the GPU arm fails loudly (non-zero exit, no JSON
line) when no GPU is present instead of falling back to the CPU."""

import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _run(*args, timeout=600):
    env = dict(os.environ, CUDA_VISIBLE_DEVICES=os.environ.get("CUDA_VISIBLE_DEVICES", ""))
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=timeout)


def _json_lines(out):
    return [json.loads(x) for x in out.splitlines() if x.strip().startswith("{")]


def test_reference_arm_prints_one_complete_line():
    import bench
    r = _run("--impl", "reference", "--workload", "C1", "--steps", "2", "--warmup", "1")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 1
    assert d["higher_is_better"] is True and d["scaling"] in ("weak", "strong")
    assert d["vs_baseline"] is None and d["data"] == "synthetic" and d["dtype"] == "f64"
    assert d["config"]["workload"].startswith("C1")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["unit"] == d["unit"]
    assert cb["cores"] >= 1 and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


@pytest.mark.skipif(bool(os.environ.get("CUDA_VISIBLE_DEVICES")) or os.path.exists("/dev/nvidia0"),
                    reason="needs a machine without a GPU")
def test_gpu_arm_fails_loudly_without_a_gpu():
    r = _run("--workload", "C1", "--steps", "1", "--warmup", "3", "--no-cpu-baseline", "--no-e2e")
    assert r.returncode != 0
    assert _json_lines(r.stdout) == []
