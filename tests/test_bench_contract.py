"""Host-side checks of bench.py (no GPU): the reference arm, which times the
oracle on the host cores, prints one JSON line with the contract's keys; the
DRAM-traffic figure of the roofline is taken from the committed ncu ratio only
while the Dslash sources still hash to the captured ones."""
import hashlib
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 1
    assert d["higher_is_better"] is False and d["unit"] == "s/source" and d["value"] > 0
    assert "workload" in d["config"] and "model" not in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


@pytest.mark.parametrize("summary,sources,kernel", [
    ("dslash_traffic.txt", ("dslash.cuh", "tm_core.cuh"), "dslash.f16.out"),
    ("dslash_il_traffic.txt", ("dslash_il.cu", "il_core.cuh", "tm_core.cuh"), "dslash.f16il.out")])
def test_traffic_ratio_applies_only_to_the_captured_sources(summary, sources, kernel):
    sys.path.insert(0, ROOT)
    import bench
    kv = {}
    with open(os.path.join(ROOT, "profiles", summary)) as f:
        for line in f:
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
    csrc = os.path.join(ROOT, "paper_1401_6749_gb300", "csrc")
    src = b"".join(open(os.path.join(csrc, n), "rb").read() for n in sources)
    got = bench._traffic_per_launch(1_000_000, kernel)
    if hashlib.sha256(src).hexdigest() == kv["kernel_sources_sha256"]:
        assert got == round(float(kv["traffic_per_algorithmic_byte"]) * 1_000_000)
    else:
        assert got is None
