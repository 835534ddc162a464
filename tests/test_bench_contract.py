"""The reference arm of bench.py (the FP64 oracle on the host cores) keeps the
JSON-line contract and reports the same workload configuration as the GPU arm."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    res = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "3"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [l for l in res.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, res.stdout[-2000:]
    out = json.loads(lines[0])
    assert out["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in out, key
    assert out["steps"] == 2 and out["warmup"] == 3 and out["n_gpus"] == 1
    assert out["value"] > 0 and out["unit"] == "images/s" and out["higher_is_better"] is True
    assert out["cpu_baseline"]["kind"] == "oracle" and out["cpu_baseline"]["value"] == out["value"]
    assert out["cpu_baseline"]["cores"] >= 1
    assert out["e2e"] == {"value": out["value"], "unit": "images/s", "h2d_bytes_per_step": 0,
                          "d2h_bytes_per_step": 0}
    sys.path.insert(0, ROOT)
    import bench
    from synth import workloads
    assert out["metric"] == bench.METRIC
    assert out["config"] == bench._fused_config(workloads.fused_512(), 1)
