"""bench.py's host-side contract, without a GPU: the reference arm (the FP64 oracle timed on
the host cores on a bounded sample of the tabletop workload) prints one JSON line with the
keys, metric and unit of the GPU arm's line; under a multi-rank launch only rank 0 runs it;
and the committed DRAM-traffic record of the fused score kernel belongs to the current
kernel source."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _run(extra_env=None, *args):
    env = dict(os.environ)
    env.update(extra_env or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args],
                          capture_output=True, text=True, env=env, timeout=600, cwd=ROOT)


@pytest.fixture(scope="module")
def ref_line(orc):  # the oracle fixture builds the oracle library first
    r = _run(None, "--steps", "2", "--warmup", "1", "--ref-seconds", "1.5")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    return json.loads(lines[0])


def test_reference_line_keys_and_units(ref_line):
    import bench
    d = ref_line
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 1
    assert d["higher_is_better"] is True and d["scaling"] == "weak" and d["vs_baseline"] is None
    assert d["dtype"] == "f64" and d["data"] == "synthetic"
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["config"]["workload"].startswith("coarse-to-fine tabletop parse")
    assert d["config"]["hyps_per_step"] == 5 * 3 * 145800
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["unit"] == bench.UNIT and cb["cores"] >= 1
    assert cb["value"] == d["value"] and "hypotheses" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_runs_on_rank_zero_only(orc):
    r = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}, "--steps", "1", "--warmup", "0",
             "--ref-seconds", "0.5")
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [l for l in r.stdout.splitlines() if l.startswith("{")]


def test_committed_traffic_record_matches_the_kernel_source():
    import bench
    rec = json.load(open(os.path.join(ROOT, "profiles", "fused_score_tabletop.json")))
    assert rec["source_hash"] == bench._kernel_source_hash()
    assert bench._committed_traffic() == rec["dram_bytes_per_launch"] > 0
    assert "--clock-control none" in rec["command"] and " -c 1 " in rec["command"]
