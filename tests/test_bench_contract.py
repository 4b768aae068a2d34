"""The benchmark's reference arm (the FP64 oracle on the host cores) keeps the
one-JSON-line contract: the metric, unit and direction of the GPU arm, a
cpu_baseline describing the run, an e2e block with no host-device bytes; under
a multi-rank launch only rank 0 prints."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra):
    env = dict(os.environ)
    env.update(env_extra)
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                         env=env, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    return [l for l in out.stdout.splitlines() if l.strip()]


def test_reference_arm_json_line():
    lines = _run({"RANK": "0", "WORLD_SIZE": "1"})
    assert len(lines) == 1
    r = json.loads(lines[0])
    sys.path.insert(0, ROOT)
    import bench
    assert r["impl"] == "reference"
    assert r["metric"] == bench.METRIC
    assert r["unit"] == "cell transmissions/s" and r["higher_is_better"] is True
    assert r["value"] > 0 and r["steps"] == 1 and r["warmup"] == 0
    assert r["dtype"] == "f64" and r["data"] == "synthetic"
    cb = r["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == r["value"]
    assert cb["unit"] == r["unit"] and cb["sample"]
    e = r["e2e"]
    assert e["value"] == r["value"] and e["unit"] == r["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    assert "workload" in r["config"]


def test_reference_arm_other_ranks_print_nothing():
    assert _run({"RANK": "1", "WORLD_SIZE": "2"}) == []
