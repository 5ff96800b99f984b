"""bench.py's reference arm (the FP64 oracle on the host cores) prints one JSON
line on the same metric, unit, direction and workload as the CUDA arm, with
its CPU-baseline and end-to-end objects."""
from __future__ import annotations

import json
import os
import subprocess
import sys

import numpy as np
import pytest

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

    class Args:
        steps, warmup = 2, 1

    # the CUDA arm prints the same config dict for the same workload and window
    assert d["config"] == bench.shared_config(w, c.nnz, Args())
    assert (d["steps"], d["warmup"], d["n_gpus"]) == (2, 1, 1)
    assert d["value"] > 0 and abs(d["ms_per_step"] - w.N / d["value"] * 1e3) <= 1e-6 * d["ms_per_step"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "objects/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_sampled_oracle_step_on_a_small_corpus():
    """The sampled reference step (used where the oracle cannot run whole
    iterations) scores a seeded sample against centroids of a balanced
    labelling and runs one whole update; its whole-iteration estimate scales
    the scoring time by N / sample."""
    sys.path.insert(0, ROOT)
    import bench
    from synth import CONFIGS, generate, init_ids

    w = CONFIGS["c1"].scaled(N=3_000, k=40)
    c = generate(w.N, w.D, w.zipf_s, w.mu, w.sigma, w.lo, w.hi, w.seed)
    ini = init_ids(w.N, w.k, w.init_seed)
    o = bench.sampled_reference_state(c, w, ini)
    off, _, _, _ = o.centroids()
    assert np.all(np.diff(off) > 0)  # every cluster of the balanced labelling has members
    meas, est = bench.sampled_oracle_step(o, w, 0)
    assert meas > 0 and est > 0
    assert not bench.oracle_is_sampled(CONFIGS["c2"]) and bench.oracle_is_sampled(CONFIGS["c5"])


def test_roofline_bound_follows_the_serving_memory():
    """The roofline names the memory that serves most of the algorithmic
    bytes: the posting structures count as L2-served when they fit in L2, and
    any rate above the HBM peak is L2-served."""
    sys.path.insert(0, ROOT)
    import bench
    from synth import CONFIGS

    w = CONFIGS["c2"]
    per = [dict(ms_assign=10.0, ms_update=1.0, postings=4e10, dense_entries=0, simcalc=w.N * w.k)]
    peaks = {"l2": 20000.0, "hbm": 6000.0}
    small, big = 100 << 20, 1 << 30
    r = bench.roofline(per, w, 57_000_000, "fp32", peaks, 6800.0, small, 0)
    assert r["bound"] == "l2" and r["peak"] == 20000.0
    alg = 57_000_000 * 8 + (w.N + 1) * 8 + w.N * 16 + w.k + 4e10 * 6
    assert r["achieved"] == pytest.approx(alg / 0.010 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 20000.0)
    # a file larger than L2 at that rate (above the HBM peak): still L2-served
    r = bench.roofline(per, w, 57_000_000, "fp32", peaks, 6800.0, big, 0)
    assert r["bound"] == "l2"
    slow = [dict(per[0], ms_assign=100.0)]
    r = bench.roofline(slow, w, 57_000_000, "fp32", peaks, 6800.0, big, 0)
    assert r["bound"] == "hbm" and r["peak"] == 6800.0
    assert r["frac"] == pytest.approx(alg / 0.100 / 1e9 / 6800.0)
    # dense rows that fit in L2 serve their bytes from L2 even when the sparse file does not fit
    per = [dict(ms_assign=10.0, ms_update=1.0, postings=3e9, dense_postings=2e9, dense_entries=4e10, simcalc=0)]
    r = bench.roofline(per, w, 57_000_000, "bf16", peaks, 6800.0, big, small)
    assert r["bound"] == "l2"
