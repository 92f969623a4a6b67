"""The benchmark's reference arm on CPU: `bench.py --impl reference` times
the FP64 oracle and prints one JSON line with the contract's keys; a rank
other than 0 prints nothing and exits 0.  Also the rule that ties the
committed ncu counters to the correlate kernel's source."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(env_extra, *args):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args],
                          capture_output=True, text=True, timeout=600, env=env, cwd=ROOT)


def test_reference_arm_prints_one_line():
    r = run_bench({}, "--impl", "reference", "--steps", "1", "--warmup", "0",
                  "--ref-templates", "2")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["config"]["templates"] == 1 << 20 and d["config"]["segment_len"] == 1 << 16


def test_reference_arm_other_ranks_exit_quietly():
    r = run_bench({"RANK": "1", "WORLD_SIZE": "2"}, "--impl", "reference", "--steps", "1",
                  "--warmup", "0", "--ref-templates", "2", "--gpus", "2")
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def test_counter_record_is_tied_to_the_source(tmp_path, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        rec = json.load(f)["correlate_kernel"]
    assert rec["dram_bytes_per_correlation"] > 16384  # at least the template itself
    assert set(rec["counters"]) >= {"sm__pipe_fma_cycles_active_pct", "smsp__issue_active_pct"}
    monkeypatch.setattr(bench, "correlate_source_hash", lambda: "0" * 64)
    assert bench.traffic_record(1 << 20) is None and bench.ncu_counters() is None
    monkeypatch.setattr(bench, "correlate_source_hash", lambda: rec["source_sha256"])
    assert bench.traffic_record(2) == 2 * rec["dram_bytes_per_correlation"]
    assert bench.ncu_counters()["smsp__issue_active_pct"] == rec["counters"]["smsp__issue_active_pct"]
