"""bench.py's reference arm (the oracle on the host cores) prints one JSON
line in the contract's shape; no GPU involved."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl",
                        "reference", "--steps", "2", "--warmup", "1",
                        "--reference-grid", "12"],
                       capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup",
              "ms_per_step", "higher_is_better", "cpu_baseline", "e2e", "config"):
        assert k in line
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["config"]["workload"] == "grid7cd_12"
    assert line["cpu_baseline"]["cores"] == line["config"]["workers"] >= 1


def test_extra_leg_failure_is_recorded_not_fatal():
    """A failing extra leg is recorded as an error and the later legs still
    run, so the bench always prints its line."""
    import bench

    def ok(a, b):
        return {"sum": a + b}

    def boom(a, b):
        raise MemoryError("out of device memory")
    extras = {}
    bench.run_legs(extras, [("first", ok), ("second", boom), ("third", ok)], 1, 2)
    assert extras["first"] == {"sum": 3} and extras["third"] == {"sum": 3}
    assert extras["second"] == {"error": "MemoryError: out of device memory"}
