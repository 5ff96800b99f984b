"""Dense head-term rows in the assignment scan.

A term whose posting list holds a large share of its instance's clusters is
read from a dense row (its value for every cluster, in scan order) into FP32
registers instead of posting by posting. The labels must not depend on that
layout: with the error bound widened by the FP32 chain and the exact
re-score, a run with dense rows gives the labels, counts and centroids of a
run without them, and both follow the FP64 oracle.
"""
from __future__ import annotations

import numpy as np
import pytest

from synth import CONFIGS
from tests.gpu_harness import corpus_for, gpu_instance, lockstep

pytestmark = pytest.mark.gpu


def _run(c, k, ini, iters, **kw):
    g = gpu_instance(c, k, ini, **kw)
    recs = []
    try:
        for _ in range(iters):
            n = g.assign()
            st = g.stats()
            recs.append((n, st["postings"], st["filtered"], st["n_moving"], st["simcalc"]))
            if st["iter"] > 1 and n == 0:
                break
            g.update()
        return recs, g.labels(), g.centroids(), g.stats()
    finally:
        g.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp16"])
@pytest.mark.parametrize("icp", [True, "relaxed", False])
def test_dense_rows_change_no_label(precision, icp):
    w = CONFIGS["c2"].scaled(N=6_000, D=6_000, k=70)
    c, ini = corpus_for(w, seed=41)
    a = _run(c, w.k, ini, 12, precision=precision, icp=icp, dense_max_bytes=-1)
    b = _run(c, w.k, ini, 12, precision=precision, icp=icp, dense_min_fraction=0.05)
    assert b[3]["dense_terms"] > 0 and b[3]["dense_entries"] > 0, "no dense row was used"
    assert a[3]["dense_terms"] == 0 and a[3]["dense_entries"] == 0
    if icp == "relaxed":
        # the relaxed test decides on error-bounded scores, and dense rows
        # widen the bound: which objects it restricts may differ, not labels
        assert [r[0] for r in a[0]] == [r[0] for r in b[0]], "changed counts differ"
    else:
        assert a[0] == b[0], "per-iteration counts differ"
    assert np.array_equal(a[1], b[1]), "labels differ"
    for x, y in zip(a[2], b[2]):
        assert np.array_equal(x, y), "centroids differ"


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_dense_rows_lockstep_with_the_oracle(precision):
    """Most of the scan from dense rows (lists of 5 % of k and up)."""
    w = CONFIGS["c2"].scaled(N=5_000, D=5_000, k=64)
    c, ini = corpus_for(w, seed=43)
    recs = lockstep(c, w.k, ini, 8, precision=precision, dense_min_fraction=0.05)
    assert any(r["stats"]["dense_entries"] > 0 for r in recs)
    assert sum(r["ties"] for r in recs) <= max(2, w.N // 1000)  # near ties (FP64 margin < 1e-6) only


def test_dense_capacity_raises_the_threshold():
    """Rows are chosen by list length relative to k (in steps of k / 64), the
    longest first, while they fit the capacity. A capacity equal to the rows
    of the lists holding at least half of the clusters makes a run that would
    take lists from 1 % of k up stop at exactly those rows; the run is still
    exact. (k = 256: lists shorter than 32 postings never get a row, so a
    smaller k would leave no list between 32 postings and k / 2.)"""
    w = CONFIGS["c2"].scaled(N=8_000, D=5_000, k=256)
    c, ini = corpus_for(w, seed=47)
    half = _run(c, w.k, ini, 8, dense_min_fraction=0.5)
    rows, terms = half[3]["dense_row_entries"], half[3]["dense_terms"]
    assert rows > 0 and terms > 0
    a = _run(c, w.k, ini, 8, dense_max_bytes=rows * 4, dense_min_fraction=0.01)
    wide = _run(c, w.k, ini, 8, dense_min_fraction=0.01)
    b = _run(c, w.k, ini, 8, dense_max_bytes=-1)
    assert wide[3]["dense_row_entries"] > rows, "the capacity must bind"
    assert a[3]["dense_row_entries"] == rows and a[3]["dense_terms"] == terms
    assert a[0] == b[0] and np.array_equal(a[1], b[1])


def test_dense_rows_with_global_score_vectors():
    w = CONFIGS["c2"].scaled(N=4_000, D=5_000, k=90)
    c, ini = corpus_for(w, seed=53)
    a = _run(c, w.k, ini, 8, score_buffer="global", dense_min_fraction=0.05)
    b = _run(c, w.k, ini, 8, score_buffer="shared", dense_max_bytes=-1)
    assert a[3]["assign_global"] == 1 and a[3]["dense_terms"] > 0
    assert a[0] == b[0] and np.array_equal(a[1], b[1])


def test_dense_rows_in_a_batch():
    """Instances of different k: each dense row has its instance's length."""
    from paper_2103_16141_gb300 import SIVFBatch
    from synth import batched_instances, generate, init_ids
    ws = batched_instances(5, scale=0.04)
    cs = [generate(w.N, w.D, w.zipf_s, w.mu, w.sigma, w.lo, w.hi, 300 + m) for m, w in enumerate(ws)]
    inis = [init_ids(w.N, w.k, 400 + m) for m, w in enumerate(ws)]
    a = SIVFBatch(cs, [w.k for w in ws], inis, precision="fp16", dense_min_fraction=0.05)
    b = SIVFBatch(cs, [w.k for w in ws], inis, precision="fp16", dense_max_bytes=-1)
    try:
        ia, oa = a.run(30)
        ib, ob = b.run(30)
        assert a.stats()["dense_terms"] > 0
        assert np.array_equal(ia, ib) and np.array_equal(oa, ob)
        for m in range(len(ws)):
            assert np.array_equal(a.labels(m), b.labels(m))
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_dense_mean_variant_equals_the_hybrid(precision):
    """dense_all: every term is read from a dense row (the centroids as a
    dense matrix in scan order, Lloyd-ICP with full-expression means). Same
    labels, method-level counts and centroids as the default layout."""
    w = CONFIGS["c2"].scaled(N=6_000, D=6_000, k=70)
    c, ini = corpus_for(w, seed=73)
    a = _run(c, w.k, ini, 12, precision=precision, dense_all=True)
    b = _run(c, w.k, ini, 12, precision=precision)
    st = a[3]
    assert st["dense_postings"] == st["postings"], "every posting from a dense row"
    assert a[0] == b[0] and np.array_equal(a[1], b[1])
    for x, y in zip(a[2], b[2]):
        assert np.array_equal(x, y)


def test_dense_mean_variant_lockstep_with_the_oracle():
    w = CONFIGS["c2"].scaled(N=4_000, D=5_000, k=60)
    c, ini = corpus_for(w, seed=79)
    recs = lockstep(c, w.k, ini, 8, dense_all=True)
    assert all(r["stats"]["dense_postings"] == r["stats"]["postings"] for r in recs)
