"""bench.py's reference arm on CPU: the FP64 oracle timed on the host cores prints one JSON
line with the keys of the benchmark contract, and ranks other than 0 exit without output."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env):
    env = dict(os.environ, **extra_env)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                           "--workload", "manufactured_64", "--steps", "1", "--warmup", "3"],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_json_line():
    r = _run({"RANK": "0"})
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == "MLUPS" and line["unit"] == "MLUPS"
    assert line["value"] > 0 and line["higher_is_better"] is True and line["steps"] == 1
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert "manufactured_64" in cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["h2d_bytes_per_step"] == 0
    assert e2e["d2h_bytes_per_step"] == 0 and e2e["unit"] == "MLUPS"
    assert line["config"]["workload"] == "manufactured_64"


def test_reference_arm_other_ranks_are_silent():
    r = _run({"RANK": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def test_cpu_full_run_reports_both_legs():
    """The opt-in full run of the small configuration (here 3 steps instead of 500): both
    thread counts, converged statuses, sweep counts and rates."""
    sys.path.insert(0, ROOT)
    import bench
    out = bench.cpu_full_run(steps=3)
    assert out["workload"] == "manufactured_64" and out["steps"] == 3
    for leg in ("all_cores", "single_thread"):
        r = out[leg]
        assert r["status"] == 0 and r["sweeps"] > 0 and r["MLUPS"] > 0 and r["seconds"] > 0
    assert out["single_thread"]["threads"] == 1
