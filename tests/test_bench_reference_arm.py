"""The benchmark's reference arm (`bench.py --impl reference`) on the host
cores: the FP64 oracle timed on a bounded sample of the benchmark workload,
printed as one JSON line with the same metric, unit and workload as the
native arm.  Under a multi-rank launch only rank 0 works and prints."""
import json
import os
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None, timeout=300):
    env = dict(os.environ)
    env.update(extra_env or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                           "--warmup", "0"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=timeout)


def test_reference_arm_prints_the_contract_line():
    p = _run()
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    j = json.loads(lines[0])
    assert j["impl"] == "reference"
    assert j["metric"] == bench.METRIC and j["unit"] == "solves/s" and j["higher_is_better"] is True
    assert j["steps"] == 1 and j["warmup"] == 0 and j["n_gpus"] == 1
    assert j["value"] > 0 and abs(j["ms_per_step"] * 1e-3 * j["value"] - 1.0) < 1e-9
    # the same workload as the native arm's default
    assert j["config"]["workload"] == bench.WORKLOADS["krr_laplace_mix"][0]
    cb = j["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == j["value"] and cb["sample"]
    e2e = j["e2e"]
    assert e2e["value"] == j["value"] and e2e["unit"] == j["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_without_work():
    p = _run({"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"}, timeout=120)
    assert p.returncode == 0, p.stderr[-2000:]
    assert not [l for l in p.stdout.splitlines() if l.startswith("{")]
