"""The benchmark's reference arm (`bench.py --impl reference`) needs no GPU: it times the FP64 oracle on
the host cores on a bounded sample of the workload and prints one JSON line.  This checks that line's
keys and their consistency (the oracle is test infrastructure; this is the one bench leg that runs it)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                         cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    r = json.loads(lines[0])
    assert r["impl"] == "reference" and r["higher_is_better"] is True
    assert r["unit"] == "particle-evals/s" and r["value"] > 0 and r["ms_per_step"] > 0
    assert r["steps"] == 1 and r["warmup"] >= 3 and r["n_gpus"] == 1
    assert r["vs_baseline"] is None and r["dtype"] == "f64"
    cb = r["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == r["value"] and cb["cores"] >= 1 and cb["sample"]
    assert r["e2e"] == {"value": r["value"], "unit": r["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert r["config"]["workload"].startswith("na_1m")
