"""The warp-per-object assignment of filtered objects.

Filtered objects (own cluster invariant) of an instance with few moving
clusters are scored by one warp each instead of one CTA each. The warp stages
the terms in the CTA kernel's chunks and forms the same dense FP32 chains and
fixed-point adds, so both paths give the same scores: the same labels, the
same counts of every iteration, the same centroids, and (through the relaxed
filter, which compares stored own scores) the same own scores. The CTA
kernel's filtered branch stays checked against the oracle with the warp path
off.
"""
from __future__ import annotations

import numpy as np
import pytest

from synth import CONFIGS
from tests.gpu_harness import corpus_for, gpu_instance, lockstep

pytestmark = pytest.mark.gpu

COUNTS = ("changed", "n_moving", "filtered", "simcalc", "postings", "dense_postings", "dense_entries", "rescored",
          "rescore_cands")


def _run(c, k, ini, iters, **kw):
    g = gpu_instance(c, k, ini, **kw)
    recs, light = [], 0
    try:
        for _ in range(iters):
            n = g.assign()
            st = g.stats()
            recs.append(tuple(st[x] for x in COUNTS))
            light += st["light_objects"]
            if st["iter"] > 1 and n == 0:
                break
            g.update()
        return recs, g.labels(), g.centroids(), light
    finally:
        g.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp16"])
@pytest.mark.parametrize("icp", [True, "relaxed"])
def test_warp_path_equals_cta_path(precision, icp):
    w = CONFIGS["c2"].scaled(N=8_000, D=8_000, k=90)
    c, ini = corpus_for(w, seed=61)
    a = _run(c, w.k, ini, 25, precision=precision, icp=icp, dense_min_fraction=0.1)
    b = _run(c, w.k, ini, 25, precision=precision, icp=icp, dense_min_fraction=0.1, light_max_moving=-1)
    assert a[3] > 0 and b[3] == 0, "the warp path must be used (and off in the second run)"
    assert a[0] == b[0], "per-iteration counts differ"
    assert np.array_equal(a[1], b[1])
    for x, y in zip(a[2], b[2]):
        assert np.array_equal(x, y)


def test_cap_on_the_moving_count():
    """With a cap of 8 moving clusters, only iterations with at most 8 moving
    clusters send objects to the warp path; the run is unchanged."""
    w = CONFIGS["c2"].scaled(N=8_000, D=8_000, k=90)
    c, ini = corpus_for(w, seed=67)
    g = gpu_instance(c, w.k, ini, light_max_moving=8)
    try:
        for _ in range(25):
            n = g.assign()
            st = g.stats()
            if st["light_objects"]:
                assert st["n_moving_prev"] <= 8
            if st["iter"] > 1 and n == 0:
                break
            g.update()
    finally:
        g.close()
    a = _run(c, w.k, ini, 25, light_max_moving=8)
    b = _run(c, w.k, ini, 25, light_max_moving=-1)
    assert a[0] == b[0] and np.array_equal(a[1], b[1])


def test_cta_filtered_branch_against_the_oracle():
    """The CTA kernel's front scan of filtered objects (warp path off)."""
    w = CONFIGS["c2"].scaled(N=5_000, D=6_000, k=70)
    c, ini = corpus_for(w, seed=71)
    recs = lockstep(c, w.k, ini, 12, light_max_moving=-1)
    assert any(r["stats"]["filtered"] > 0 for r in recs)
    assert all(r["stats"]["light_objects"] == 0 for r in recs)


def test_warp_path_in_a_batch():
    from paper_2103_16141_gb300 import SIVFBatch
    from synth import batched_instances, generate, init_ids
    ws = batched_instances(6, scale=0.04)
    cs = [generate(w.N, w.D, w.zipf_s, w.mu, w.sigma, w.lo, w.hi, 500 + m) for m, w in enumerate(ws)]
    inis = [init_ids(w.N, w.k, 600 + m) for m, w in enumerate(ws)]
    a = SIVFBatch(cs, [w.k for w in ws], inis, precision="fp16", light_max_moving=0)
    b = SIVFBatch(cs, [w.k for w in ws], inis, precision="fp16", light_max_moving=-1)
    try:
        ia, oa = a.run(40)
        ib, ob = b.run(40)
        assert np.array_equal(ia, ib) and np.array_equal(oa, ob)
        for m in range(len(ws)):
            assert np.array_equal(a.labels(m), b.labels(m))
    finally:
        a.close()
        b.close()
