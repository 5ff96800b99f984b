"""bench.py's reference arm (the FP64 oracle on the host cores) prints one JSON
line on the same metric, unit, direction and workload as the CUDA arm, with
its CPU-baseline and end-to-end objects."""
from __future__ import annotations

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line_matches_the_cuda_arm_contract():
    sys.path.insert(0, ROOT)
    import bench
    from synth import CONFIGS, generate

    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--config", "c1", "--steps", "2",
                          "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=300, check=True)
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    w = CONFIGS["c1"]
    c = generate(w.N, w.D, w.zipf_s, w.mu, w.sigma, w.lo, w.hi, w.seed)
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == "objects/s" and d["higher_is_better"] is True
    assert d["config"]["workload"] == bench.workload_name(w, c.nnz)
    assert d["config"]["icp"] == "sivf" and d["config"]["max_iter"] == w.max_iter
    assert (d["steps"], d["warmup"], d["n_gpus"]) == (2, 1, 1)
    assert d["value"] > 0 and abs(d["ms_per_step"] - w.N / d["value"] * 1e3) <= 1e-6 * d["ms_per_step"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "objects/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
