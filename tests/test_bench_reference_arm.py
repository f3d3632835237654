"""The benchmark's reference arm (the FP64 oracle on the host cores) runs without a GPU and
prints one JSON line with the keys the benchmark contract asks for."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_complete_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "box", "--steps", "2",
                        "--warmup", "1", "--cpu-budget", "1"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    # the step is the measured sample, the config names the workload as the GPU arm does
    cb = d["cpu_baseline"]
    assert abs(d["ms_per_step"] - 1e3 * cb["seconds"]) < 0.5 * d["ms_per_step"] and cb["pair_points"] > 0
    assert set(d["config"]) >= {"workload", "pairs", "frames", "pair_points_per_step", "l2", "parallelism"}
    assert "stand-in" in cb["sample"]
