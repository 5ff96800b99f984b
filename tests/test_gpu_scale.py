"""Full-size parity of the large workloads (1M x 140K, k = 10,000 and
8M x 140K, k = 20,000; BF16 postings with exact re-score).

The oracle cannot run these iterations whole, so after each assignment it
rebuilds the centroids from the GPU's previous labels (its own update step)
and scores a sample of objects one by one; the GPU labels of the sample must
equal the oracle's except where the FP64 top-2 margin is below 1e-6, and the
update objective must agree within 1e-6 relative.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import Oracle
from synth import CONFIGS
from tests.gpu_harness import OBJECTIVE_RTOL, compare_labels, corpus_for, gpu_instance, rel

pytestmark = pytest.mark.gpu


def sampled_lockstep(name, iters, sample, threads=4):
    w = CONFIGS[name]
    c, ini = corpus_for(w)
    g = gpu_instance(c, w.k, ini, precision=w.precision)
    o = Oracle(c, w.k, ini, icp=False, threads=0)
    rng = np.random.default_rng(1)
    rescored = 0
    try:
        for r in range(1, iters + 1):
            g.assign()
            st = g.stats()
            rescored += st["rescored"]
            lab = g.labels()
            ids = np.sort(rng.choice(w.N, size=sample, replace=False))
            lab_o, best, second = o.score_objects(ids)
            compare_labels(lab[ids], lab_o, best, second, f"{name} iteration {r}")
            o.set_labels(lab)
            u = o.update()
            g.update()
            assert rel(g.stats()["objective_update"], u.objective) <= OBJECTIVE_RTOL
    finally:
        g.close()
    return rescored


def test_c3_bf16_iterations_1_to_3_against_oracle():
    sampled_lockstep("c3", iters=3, sample=2000)


def test_c5_bf16_iterations_1_to_2_against_oracle():
    sampled_lockstep("c5", iters=2, sample=1000)
