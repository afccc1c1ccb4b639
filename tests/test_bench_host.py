"""bench.py's reference arm (the FP64 oracle on the host cores) prints one
JSON line with the keys of the benchmark contract, for the workload it was
asked for (runs without a GPU; a small corpus keeps it to seconds)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

KEYS = ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
        "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e")


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--n", "1500", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    d = json.loads(lines[0])
    for key in KEYS:
        assert key in d, key
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 1
    assert d["config"]["n"] == 1500 and d["config"]["N"] == 4096 and d["config"]["k"] == 50
    assert d["value"] > 0 and d["higher_is_better"] is True and d["unit"] == "pair-estimates/s"
    # one step = all 1500 x 1499 ordered pairs at the measured rate
    assert abs(d["ms_per_step"] - 1500 * 1499 / d["value"] * 1e3) <= 1e-6 * d["ms_per_step"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert "1,500 rows" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    # the seconds the oracle actually ran are reported beside the extrapolation
    assert d["timed_s"] > 0 and abs(d["timed_ms_per_step"] - d["timed_s"] * 1e3) <= 1e-6 * d["timed_s"] * 1e3
