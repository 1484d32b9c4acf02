"""The reference arm of bench.py on the host (no GPU): the oracle, as it stands, timed on one bounded
sample per step, printed as one JSON line of the bench contract with impl = "reference"."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1
    assert d["unit"] == "solves/s" and d["higher_is_better"] is True and d["value"] > 0
    # one step is one bounded sample: its wall time, and the 128^3 solve time it stands for
    assert 0 < d["ms_per_step"] < d["extrapolated_ms_per_solve"]
    assert abs(d["value"] - 1e3 / d["extrapolated_ms_per_solve"]) <= 1e-9 * d["value"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["n"] == 128 and d["config"]["tol"] == 1e-10
