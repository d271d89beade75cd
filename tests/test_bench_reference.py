"""The benchmark's reference arm (the CPU oracle timed on the host cores) on
the CPU: one JSON line with the fields the measurement contract needs, and
silence on every rank but 0."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CMD = [sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3",
       "--slots", str(1 << 20)]


def run(extra_env=None, args=()):
    env = dict(os.environ)
    env.update(extra_env or {})
    return subprocess.run(CMD + list(args), cwd=ROOT, env=env, capture_output=True, text=True,
                          timeout=600)


def test_reference_line():
    r = run()
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == "Gops/s insert/find/mixed at 95% load" and d["unit"] == "Gops/s"
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["ms_per_step"] > 0 and d["vs_baseline"] is None
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert cb["unit"] == "Gops/s" and cb["sample"]
    assert cb["host"]["cpus"] == os.cpu_count() and cb["host"]["model"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    c = d["config"]
    assert c["slots"] == 1 << 20 and c["n_insert"] == (1 << 20) * 19 // 20
    assert "fits in the 129 MB L2" in c["l2"]


def test_other_ranks_print_nothing():
    r = run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}, ["--gpus", "2"])
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""
