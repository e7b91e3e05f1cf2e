"""The benchmark's reference arm (the FP64 oracle timed on the host) keeps
the JSON-line contract: one line with the arm's metric, unit and config, a
cpu_baseline object describing the run and an e2e object with no transfers;
ranks other than 0 print nothing and exit 0."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra):
    env = dict(os.environ)
    env.update(env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                           "--steps", "1", "--warmup", "0"],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_line():
    r = _run({"RANK": "0"})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == d["unit"] == "walker-steps/s"
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 0
    assert d["config"]["workload"].startswith("rand100x2000")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_other_ranks_are_silent():
    r = _run({"RANK": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def test_feasibility_flags():
    # Every leg carrying max_violation gets a "feasible" flag from its measured
    # and audited violations (bound 1e-6 |b|_inf, |b|_inf = 1 here).
    sys.path.insert(0, ROOT)
    import bench
    line = {"feasibility": {"max_violation": -3e-5, "audit": {"run_max_violation": -1e-5}},
            "batched": {"max_violation": -2e-5, "audit": {"run_max_violation": 2e-6}},
            "other": {"x": {"max_violation": 5e-7, "run_max_violation": -1.0}}}
    assert bench.mark_feasibility(line) is False
    assert line["feasibility"]["feasible"] is True
    assert line["batched"]["feasible"] is False
    assert line["other"]["x"]["feasible"] is True
