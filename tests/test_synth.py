"""The seeded input generator (shared by the oracle and the CUDA path, and
holding none of the method's arithmetic) against the recipe it documents:
CSR well-formed, terms ascending and distinct in each row, values positive
and rows of unit L2 norm, lengths inside their clip range, a Zipf head,
determinism by seed, and the nnz that the configuration table records."""
from __future__ import annotations

import numpy as np
import pytest

from synth import CONFIGS, batched_instances, generate, init_ids


def corpus(name):
    w = CONFIGS[name]
    return w, generate(w.N, w.D, w.zipf_s, w.mu, w.sigma, w.lo, w.hi, w.seed)


@pytest.mark.parametrize("name", ["c1", "c5s"])
def test_csr_is_well_formed_and_rows_are_unit_vectors(name):
    w, c = corpus(name)
    rp, idx, val = c.row_ptr, c.idx, c.val
    assert rp.dtype == np.int64 and idx.dtype == np.int32 and val.dtype == np.float32
    assert rp[0] == 0 and rp[-1] == len(idx) == len(val)
    assert np.all(np.diff(rp) >= 0)
    assert idx.min() >= 0 and idx.max() < w.D
    # terms strictly ascending inside every row (distinct terms)
    d = np.diff(idx.astype(np.int64))
    row_start = np.zeros(len(idx), dtype=bool)
    row_start[rp[:-1][np.diff(rp) > 0]] = True
    assert np.all(d[~row_start[1:]] > 0)
    assert np.all(np.isfinite(val)) and np.all(val > 0)
    norms = np.sqrt(np.add.reduceat(val.astype(np.float64) ** 2, rp[:-1][np.diff(rp) > 0]))
    assert np.max(np.abs(norms - 1.0)) < 1e-6
    # distinct terms per row never exceed the clipped token count
    assert np.diff(rp).max() <= w.hi


def test_nnz_matches_the_recorded_configurations():
    # the "measured nnz" column of the configuration table
    assert corpus("c1")[1].nnz == 79_447
    assert corpus("c5s")[1].nnz == 29_995_894


def test_generation_is_deterministic_by_seed():
    w = CONFIGS["c1"]
    a = generate(w.N, w.D, w.zipf_s, w.mu, w.sigma, w.lo, w.hi, w.seed)
    b = generate(w.N, w.D, w.zipf_s, w.mu, w.sigma, w.lo, w.hi, w.seed)
    c = generate(w.N, w.D, w.zipf_s, w.mu, w.sigma, w.lo, w.hi, w.seed + 1)
    assert np.array_equal(a.row_ptr, b.row_ptr) and np.array_equal(a.idx, b.idx) and np.array_equal(a.val, b.val)
    assert not (np.array_equal(a.row_ptr, c.row_ptr) and np.array_equal(a.idx, c.idx))


def test_document_frequencies_have_a_zipf_head():
    # Zipf(s) over ranks with a seeded permutation to term ids: sorted by
    # document frequency, the head terms appear in far more documents than
    # the median term, and the frequencies fall with rank
    w, c = corpus("c5s")
    df = np.sort(np.bincount(c.idx, minlength=w.D))[::-1]
    assert df[0] > 0.5 * w.N          # the top term is in most documents
    assert df[0] > 50 * max(df[w.D // 2], 1)
    top = df[:1000].astype(np.float64)
    slope = np.polyfit(np.log(np.arange(10, 1000)), np.log(top[9:999]), 1)[0]
    assert -1.3 < slope < -0.3         # a power-law fall, flattened at the top by distinct terms


def test_init_ids_are_distinct_seeded_documents():
    a = init_ids(10_000, 500, 7)
    b = init_ids(10_000, 500, 7)
    assert np.array_equal(a, b)
    assert len(np.unique(a)) == 500 and a.min() >= 0 and a.max() < 10_000
    assert not np.array_equal(a, init_ids(10_000, 500, 8))
    assert sorted(init_ids(50, 50, 3).tolist()) == list(range(50))  # k = N: every document once
    with pytest.raises(ValueError):
        init_ids(10, 11, 1)


def test_batched_instances_follow_their_stated_ranges():
    ws = batched_instances(64)
    assert len(ws) == 64 and [w.seed for w in ws] == list(range(64))
    for w in ws:
        assert 5_000 <= w.N <= 200_000
        assert 20_000 <= w.D <= 100_000
        assert 16 <= w.k <= 2_000 and w.k <= w.N
        assert w.precision == "fp16"
    small = batched_instances(6, scale=0.05)
    assert all(w.k <= w.N for w in small)
