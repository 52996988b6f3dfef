"""The benchmark runs end to end on the GPU and prints the one JSON line its
contract asks for: the headline metric with roofline, e2e, clocks and launch
count, the CPU baseline left out here, and every form (few steps each)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_prints_the_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--steps", "3", "--warmup", "3",
                        "--form-steps", "3", "--no-cpu-baseline"],
                       cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "gpu_launches", "clocks"):
        assert k in d, k
    assert d["value"] > 0 and d["unit"] == "MLUPS" and d["steps"] == 3 and d["n_gpus"] == 1
    roof = d["roofline"]
    assert roof["bound"] == "hbm" and 0 < roof["frac"] < 1.5 and roof["peak"] > 0
    assert d["e2e"]["value"] > 0 and d["e2e"]["h2d_bytes_per_step"] > 0
    assert d["gpu_launches"] == 3 * 3
    assert "workload" in d["config"]
    forms = d["forms"]
    for k in ("f32", "mdf3", "deterministic", "eq3", "school", "free_sphere", "adjoint", "f16", "bf16", "aa",
              "aa_f16", "large_sphere", "batched"):
        assert k in forms, k
    for k in ("f16", "bf16", "school", "batched"):
        assert forms[k]["value"] > 0, k


def test_bench_single_form():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--form", "batched", "--batch-envs", "3",
                        "--steps", "3", "--warmup", "3", "--variant", "plain"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    d = json.loads([l for l in r.stdout.splitlines() if l.startswith("{")][-1])
    assert d["form"] == "batched" and d["envs"] == 3 and d["value"] > 0
