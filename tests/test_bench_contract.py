"""The bench's JSON contract, checked on the host: the reference arm (the
FP64 oracle timed on the CPU) runs on a small grid and prints one line with
the keys the comparison needs, and its metric and config are the ones the
GPU arm reports for the same workload."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_comparable_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--nx", "32", "--ny", "16", "--k", "4", "--steps", "2", "--warmup", "1"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 1 and d["unit"] == "frequencies/s"
    for key in ("value", "unit", "cores", "kind", "sample"):
        assert key in d["cpu_baseline"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    sys.path.insert(0, ROOT)
    import bench
    import workloads as W
    g = W.ns_grid(32, 16)
    assert d["metric"] == bench.metric_name(g, 4)
    assert d["config"] == bench.workload_config(g, 4, 1)
