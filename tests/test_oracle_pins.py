"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test below checks the oracle against something other than itself:
  * the plain definition rho_ij = <x_i, mu_j> by dense brute force (bit-exact);
  * closed forms (k = 1; k = N; block-orthogonal corpora; a hand-worked case);
  * the ICP invariant: the filtered run (Algorithm 4) makes exactly the
    assignments of the unfiltered run (Algorithm 2) from the same start
    (Section 2.1 / Section 3.2: ICP only skips similarities whose outcome is
    already known);
  * the count identities of Section 6 (IVF computes all N*k similarities; SIVF
    computes #moving for a filtered object and k otherwise);
  * spherical k-means theory (Section 1): the objective sum of cosines never
    decreases, and after an update sum_{i in C_j} <x_i, mu_j> = ||s_j||;
  * the layout of Algorithm 5 (front = moving, back = invariant, ascending ids).
"""
from __future__ import annotations

import math

import numpy as np
import pytest

from oracle import Oracle
from synth import CONFIGS, generate, init_ids
from synth.corpus import from_dense
from tests.helpers import brute_force_scores, mean_direction, random_dense_corpus

SMALL_SEEDS = list(range(8))


def _small(seed, N=36, D=24, k=5, dup=3, density=0.25):
    X, c = random_dense_corpus(N, D, density, seed, dup_rows=dup)
    ini = init_ids(N, k, 1000 + seed)
    return X, c, ini


@pytest.mark.parametrize("seed", SMALL_SEEDS)
@pytest.mark.parametrize("icp", [False, True])
def test_assignment_equals_dense_brute_force(seed, icp):
    """Algorithm 2/4 scores and labels equal the dense definition bit for bit,
    at every iteration, including exact ties from duplicated documents."""
    pin_brute_force(seed, icp)


def pin_brute_force(seed, icp, lib=None):
    X, c, ini = _small(seed)
    o = Oracle(c, 5, ini, icp=icp, lib=lib)
    for _ in range(12):
        M = o.dense_centroids()
        lab_bf, rho = brute_force_scores(X, M)
        a = o.assign()
        lab = o.labels()
        best, second, filt = o.scores()
        assert np.array_equal(lab, lab_bf)
        assert np.array_equal(best, rho[np.arange(c.N), lab_bf])
        unf = filt == 0
        srt = np.sort(rho, axis=1)
        assert np.array_equal(second[unf], srt[unf, -2])
        if a.r > 1 and a.changed == 0:
            break
        o.update()


@pytest.mark.parametrize("seed", SMALL_SEEDS[:4])
def test_score_objects_equals_dense_brute_force(seed):
    """The per-object scoring used for sampled checks at full size (Algorithm 2
    scoring without state change) equals the dense definition bit for bit:
    label (lowest index on ties), best and second-best score, for objects in
    any order, against seed centroids holding an exact tie (two identical
    documents) and against updated centroids."""
    pin_score_objects(seed)


def pin_score_objects(seed, lib=None):
    X, c, _ = _small(seed)
    ini = np.array([0, c.N - 1, 5, 9, 14], dtype=np.int32)  # rows 0 and N-1 are identical
    o = Oracle(c, 5, ini, icp=True, lib=lib)
    ids = np.random.default_rng(seed).permutation(c.N).astype(np.int64)
    for step in range(3):
        lab_bf, rho = brute_force_scores(X, o.dense_centroids())
        lab, best, second = o.score_objects(ids)
        assert np.array_equal(lab, lab_bf[ids])
        assert np.array_equal(best, rho[ids, lab_bf[ids]])
        assert np.array_equal(second, np.sort(rho, axis=1)[ids, -2])
        if step == 0:
            assert np.any(rho[:, 0] == rho[:, 1]) and lab_bf[0] == 0 and lab_bf[c.N - 1] == 0
        o.assign()
        o.update()


@pytest.mark.parametrize("seed", SMALL_SEEDS)
def test_update_is_normalised_mean_of_members(seed):
    """Algorithm 5 lines 17-20 then unit length: mu_j = s_j / ||s_j||, support =
    union of member terms, ||mu_j|| = 1; an empty cluster keeps its centroid."""
    pin_update(seed)


def pin_update(seed, lib=None):
    X, c, ini = _small(seed)
    o = Oracle(c, 5, ini, icp=True, lib=lib)
    for _ in range(6):
        o.assign()
        M_prev = o.dense_centroids()
        lab = o.labels()
        u = o.update()
        off, term, val, snorm = o.centroids()
        M = o.dense_centroids()
        obj = 0.0
        for j in range(5):
            mem = np.nonzero(lab == j)[0]
            if len(mem) == 0:
                assert np.array_equal(M[j], M_prev[j])
                assert snorm[j] == 0.0
                continue
            ref = mean_direction(X, mem)
            np.testing.assert_allclose(M[j], ref, rtol=0, atol=1e-14)
            support = np.nonzero(X[mem].sum(axis=0))[0]
            assert np.array_equal(term[off[j]:off[j + 1]], support)
            assert abs(math.sqrt((val[off[j]:off[j + 1]] ** 2).sum()) - 1.0) <= 1e-12
            s = X[mem].astype(np.float64).sum(axis=0)
            assert abs(snorm[j] - math.sqrt((s * s).sum())) <= 1e-12 * snorm[j]
            # sum over members of <x_i, mu_j> equals ||s_j||
            assert abs(float((X[mem].astype(np.float64) @ M[j]).sum()) - snorm[j]) <= 1e-12 * snorm[j]
            obj += snorm[j]
        assert abs(u.objective - obj) <= 1e-12 * obj


def test_empty_cluster_keeps_previous_centroid():
    X, c, ini = _small(3, k=5)
    o = Oracle(c, 5, ini, icp=True)
    o.assign()
    o.update()
    M_before = o.dense_centroids()
    lab = o.labels().copy()
    lab[lab == 2] = 0  # empty cluster 2
    o.set_labels(lab)
    lam = o.lam()
    assert lam[2] == 0 or not (o.labels() == 2).any()
    u = o.update()
    assert u.empty >= 1
    assert np.array_equal(o.dense_centroids()[2], M_before[2])


@pytest.mark.parametrize("seed", SMALL_SEEDS[:4])
def test_structured_inverted_file_layout(seed):
    """Front part = centroids with lambda = 0 (moving), back = lambda = 1,
    ascending centroid id in each part, values equal to the centroid rows."""
    pin_layout(seed)


def pin_layout(seed, lib=None):
    X, c, ini = _small(seed)
    o = Oracle(c, 5, ini, icp=True, lib=lib)
    for _ in range(5):
        o.assign()
        o.update()
        lam = o.lam()
        M = o.dense_centroids()
        off, mf0, cid, uu = o.inverted_file()
        for p in range(c.D):
            seg = cid[off[p]:off[p + 1]]
            vals = uu[off[p]:off[p + 1]]
            holders = np.nonzero(M[:, p])[0]
            front = holders[lam[holders] == 0]
            back = holders[lam[holders] == 1]
            assert mf0[p] == len(front)
            assert np.array_equal(seg, np.concatenate([front, back]))
            assert np.array_equal(vals, M[seg, p])


def test_k1_closed_form():
    X, c, _ = _small(5, N=30, k=1, dup=0)
    o = Oracle(c, 1, np.array([7], dtype=np.int32), icp=True)
    hist = o.run(10)
    assert len(hist) == 2 and hist[-1][0].changed == 0
    s = X.astype(np.float64).sum(axis=0)
    mu = s / np.linalg.norm(s)
    np.testing.assert_allclose(o.dense_centroids()[0], mu, rtol=0, atol=1e-14)
    assert abs(hist[0][1].objective - np.linalg.norm(s)) <= 1e-12 * np.linalg.norm(s)
    # r = 2 objective: sum_i <x_i, mu> = ||s||
    assert abs(hist[1][0].objective - np.linalg.norm(s)) <= 1e-12 * np.linalg.norm(s)


def test_k_equals_n_each_document_its_own_cluster():
    X, c, _ = _small(11, N=25, D=40, k=25, dup=0, density=0.3)
    perm = np.random.default_rng(0).permutation(25).astype(np.int32)
    o = Oracle(c, 25, perm, icp=True)
    hist = o.run(10)
    lab = o.labels()
    assert np.array_equal(perm[lab], np.arange(25))
    assert len(hist) == 2
    norms = np.linalg.norm(X.astype(np.float64), axis=1)
    assert abs(hist[0][1].objective - norms.sum()) <= 1e-12 * 25


def test_block_orthogonal_corpus_recovers_blocks():
    rng = np.random.default_rng(4)
    k, per, width = 4, 9, 7
    X = np.zeros((k * per, k * width), dtype=np.float64)
    for b in range(k):
        for t in range(per):
            row = b * per + t
            m = rng.random(width) < 0.6
            m[rng.integers(width)] = True
            X[row, b * width:(b + 1) * width][m] = rng.random(m.sum()) + 0.1
    X /= np.linalg.norm(X, axis=1, keepdims=True)
    order = rng.permutation(len(X))
    X = X[order].astype(np.float32)
    block = (order // per).astype(np.int32)
    c = from_dense(X)
    ini = np.array([np.nonzero(block == b)[0][0] for b in range(k)], dtype=np.int32)
    o = Oracle(c, k, ini, icp=True)
    hist = o.run(10)
    assert np.array_equal(o.labels(), block)
    assert len(hist) == 2


def test_hand_worked_example():
    """Four documents, k = 2, seeds {x0, x2} (worked by hand):
    r = 1 assigns {x0, x1} -> 0 and {x2, x3} -> 1 with J = 2 + a + b;
    s0 = (1+a, b, 0, 0), s1 = (0, 0, 1+b, a); the update objective is
    ||s0|| + ||s1||; r = 2 changes nothing."""
    pin_hand_example()


def pin_hand_example(lib=None):
    a, b = float(np.float32(0.6)), float(np.float32(0.8))
    X = np.array([[1, 0, 0, 0], [a, b, 0, 0], [0, 0, 1, 0], [0, 0, b, a]], dtype=np.float32)
    c = from_dense(X)
    o = Oracle(c, 2, np.array([0, 2], dtype=np.int32), icp=True, lib=lib)
    a1 = o.assign()
    assert list(o.labels()) == [0, 0, 1, 1]
    assert abs(a1.objective - (2 + a + b)) <= 1e-15
    u1 = o.update()
    n0, n1 = math.sqrt((1 + a) ** 2 + b ** 2), math.sqrt((1 + b) ** 2 + a ** 2)
    assert abs(u1.objective - (n0 + n1)) <= 1e-14
    M = o.dense_centroids()
    np.testing.assert_allclose(M[0], [(1 + a) / n0, b / n0, 0, 0], rtol=0, atol=1e-15)
    np.testing.assert_allclose(M[1], [0, 0, (1 + b) / n1, a / n1], rtol=0, atol=1e-15)
    a2 = o.assign()
    assert a2.changed == 0 and list(o.labels()) == [0, 0, 1, 1]
    assert abs(a2.objective - (n0 + n1)) <= 1e-14


def _lockstep_icp_vs_ivf(c, k, ini, max_iter, lib=None):
    f = Oracle(c, k, ini, icp=True, lib=lib)
    g = Oracle(c, k, ini, icp=False, lib=lib)
    rows = []
    for _ in range(max_iter):
        off, mf0, cid, _u = f.inverted_file()
        lam_prev = f.lam()
        lab_prev = f.labels()
        af, ag = f.assign(), g.assign()
        assert np.array_equal(f.labels(), g.labels())
        bf, _, filt = f.scores()
        bg, _, _ = g.scores()
        assert np.array_equal(bf, bg)
        assert np.array_equal(f.lam(), g.lam())
        assert af.changed == ag.changed and af.objective == ag.objective
        rows.append((af, ag, off, mf0, lam_prev, lab_prev, filt))
        if af.r > 1 and af.changed == 0:
            break
        uf, ug = f.update(), g.update()
        assert uf.objective == ug.objective
    return rows


def _check_counts(c, k, rows):
    lens = np.diff(c.row_ptr)
    obj = np.repeat(np.arange(c.N), lens)
    for af, ag, off, mf0, lam_prev, lab_prev, filt in rows:
        mf = np.diff(off)
        # IVF: all N*k similarities; postings = sum over object terms of mf
        assert ag.simcalc == c.N * k
        assert ag.postings == int(mf[c.idx].sum())
        # SIVF: object filtered iff its previous cluster was invariant
        exp_f = np.zeros(c.N, dtype=bool)
        if af.r >= 2:
            exp_f = (lab_prev >= 0) & (lam_prev[np.maximum(lab_prev, 0)] == 1)
        assert np.array_equal(filt.astype(bool), exp_f)
        nmov = int((lam_prev == 0).sum())
        assert af.simcalc == int(np.where(exp_f, nmov, k).sum())
        per = np.where(exp_f[obj], mf0[c.idx], mf[c.idx])
        assert af.postings == int(per.sum())
        assert af.postings <= ag.postings
        if af.r <= 2:
            assert af.filtered == 0


@pytest.mark.parametrize("seed", SMALL_SEEDS)
def test_icp_invariant_and_counts_small(seed):
    pin_icp_counts(seed)


def pin_icp_counts(seed, lib=None):
    X, c, ini = _small(seed, N=60, D=30, k=6)
    rows = _lockstep_icp_vs_ivf(c, 6, ini, 30, lib=lib)
    _check_counts(c, 6, rows)


@pytest.mark.parametrize("seed", SMALL_SEEDS)
def test_cbicp_equals_ivf_labels_and_sivf_simcalcs(seed):
    """IVF-CBICP (Algorithm 3) traverses every posting like IVF but, for the
    filtered objects, accumulates only moving centroids like SIVF: its scores
    and labels equal both at every iteration, its sim-calcs equal SIVF's and
    its postings traversed equal IVF's."""
    pin_cbicp(seed)


def pin_cbicp(seed, lib=None):
    X, c, ini = _small(seed, N=60, D=30, k=6)
    f = Oracle(c, 6, ini, icp=True, lib=lib)
    g = Oracle(c, 6, ini, icp=False, lib=lib)
    h = Oracle(c, 6, ini, icp="cbicp", lib=lib)
    saw_filter = False
    for _ in range(30):
        af, ag, ah = f.assign(), g.assign(), h.assign()
        assert np.array_equal(h.labels(), g.labels())
        bh, sh, _ = h.scores()
        bf, sf, _ = f.scores()
        assert np.array_equal(bh, bf) and np.array_equal(sh, sf)  # best and runner-up, bit for bit
        assert ah.simcalc == af.simcalc and ah.filtered == af.filtered
        assert ah.postings == ag.postings
        assert ah.changed == ag.changed and ah.objective == af.objective
        saw_filter |= ah.filtered > 0
        if ah.r > 1 and ah.changed == 0:
            break
        f.update(), g.update(), h.update()
    return saw_filter


def test_cbicp_filters_on_c1():
    w = CONFIGS["c1"]
    c = generate(w.N, w.D, w.zipf_s, w.mu, w.sigma, w.lo, w.hi, w.seed)
    ini = init_ids(w.N, w.k, w.init_seed)
    h = Oracle(c, w.k, ini, icp="cbicp")
    f = Oracle(c, w.k, ini, icp=True)
    g = Oracle(c, w.k, ini, icp=False)
    filtered = 0
    for _ in range(w.max_iter):
        ah, af, ag = h.assign(), f.assign(), g.assign()
        assert np.array_equal(h.labels(), f.labels())
        assert ah.simcalc == af.simcalc and ah.postings == ag.postings
        filtered += ah.filtered
        if ah.r > 1 and ah.changed == 0:
            break
        h.update(), f.update(), g.update()
    assert filtered > 0


RELAXED_CASES = [(3000, 3000, 30, 31), (2000, 1000, 25, 33), (4000, 2000, 20, 31)]


@pytest.mark.parametrize("case", range(len(RELAXED_CASES)))
def test_relaxed_filter_keeps_ivf_labels(case):
    """The relaxed filter (an object whose own cluster moved keeps to the moving
    centroids when its own similarity did not decrease) gives IVF's labels and
    best scores at every iteration; it filters every object SIVF filters, and
    each object it filters in addition has a best score no lower than at the
    previous iteration."""
    assert pin_relaxed(case) > 0


def _own_similarity(c, lab, M, ids):
    """FP64 <x_i, mu_lab(i)> summed term by term in row order (the scan's order)."""
    out = np.empty(len(ids))
    for n, i in enumerate(ids):
        acc = 0.0
        for h in range(c.row_ptr[i], c.row_ptr[i + 1]):
            acc += float(c.val[h]) * M[lab[i], c.idx[h]]
        out[n] = acc
    return out


def pin_relaxed(case, lib=None):
    N, D, k, seed = RELAXED_CASES[case]
    w = CONFIGS["c1"].scaled(N=N, D=D, k=k)
    c = generate(w.N, w.D, w.zipf_s, w.mu, w.sigma, w.lo, w.hi, seed)
    ini = init_ids(w.N, w.k, seed)
    f = Oracle(c, w.k, ini, icp=True, lib=lib)
    g = Oracle(c, w.k, ini, icp=False, lib=lib)
    h = Oracle(c, w.k, ini, icp="relaxed", lib=lib)
    extra = 0
    prev_best = None
    for _ in range(40):
        # the rule, from the paper's statement: an object of a moving cluster
        # is restricted iff its similarity to its own centroid did not drop
        lab_prev, lam_prev = h.labels(), h.lam()
        eligible = np.zeros(w.N, dtype=bool)
        if prev_best is not None and 2 * int((lam_prev == 0).sum()) <= w.k:
            eligible = lam_prev[lab_prev] == 0
        ids = np.nonzero(eligible)[0]
        rise = _own_similarity(c, lab_prev, h.dense_centroids(), ids) >= prev_best[ids] if len(ids) else None
        af, ag, ah = f.assign(), g.assign(), h.assign()
        if len(ids):
            assert np.array_equal(h.scores()[2][ids].astype(bool), rise)
        assert np.array_equal(h.labels(), g.labels())
        bh, _, fh = h.scores()
        bg, _, _ = g.scores()
        _, _, ff = f.scores()
        assert np.array_equal(bh, bg)
        assert np.all(fh >= ff)
        more = (fh > ff)
        if prev_best is not None:
            assert np.all(bh[more] >= prev_best[more])
        if 2 * ah.n_moving_prev > w.k:
            assert ah.filtered == af.filtered and ah.postings == af.postings
        extra += int(more.sum())
        prev_best = bh
        if ah.r > 1 and ah.changed == 0:
            break
        f.update(), g.update(), h.update()
    return extra


def test_icp_invariant_counts_and_monotone_objective_c1():
    w = CONFIGS["c1"]
    c = generate(w.N, w.D, w.zipf_s, w.mu, w.sigma, w.lo, w.hi, w.seed)
    ini = init_ids(w.N, w.k, w.init_seed)
    rows = _lockstep_icp_vs_ivf(c, w.k, ini, w.max_iter)
    _check_counts(c, w.k, rows)
    assert any(r[0].filtered > 0 for r in rows)


@pytest.mark.parametrize("seed", [21, 22, 23])
def test_monotone_objective(seed):
    """Spherical k-means never decreases sum_i cos(x_i, mu_a(i)): the update
    objective is >= the assignment objective of the same iteration, and the
    next assignment's is >= the update's."""
    pin_monotone(seed)


def pin_monotone(seed, lib=None):
    w = CONFIGS["c1"].scaled(N=800, D=3000, k=20)
    c = generate(w.N, w.D, w.zipf_s, w.mu, w.sigma, w.lo, w.hi, seed)
    o = Oracle(c, w.k, init_ids(w.N, w.k, seed), icp=True, lib=lib)
    prev_u = None
    for _ in range(30):
        a = o.assign()
        if prev_u is not None:
            assert a.objective >= prev_u - 1e-12 * w.N
        if a.r > 1 and a.changed == 0:
            break
        u = o.update()
        assert u.objective >= a.objective - 1e-12 * w.N
        prev_u = u.objective


def test_empty_row_and_zero_scores():
    """An object sharing no term with any centroid has all-zero scores and takes
    label 0 (lowest index); an empty row behaves the same way."""
    pin_zero_scores()


def pin_zero_scores(lib=None):
    X = np.zeros((5, 6), dtype=np.float32)
    X[0, 0] = 1.0
    X[1, 1] = 1.0
    X[2, 2] = 1.0
    X[3, 5] = 1.0  # shares no term with seeds {1, 2}
    # row 4 is empty
    c = from_dense(X)
    o = Oracle(c, 2, np.array([1, 2], dtype=np.int32), icp=True, lib=lib)
    o.assign()
    lab = o.labels()
    assert lab[3] == 0 and lab[4] == 0 and lab[0] == 0
    assert lab[1] == 0 and lab[2] == 1
    hist = o.run(10)
    assert hist[-1][0].changed == 0


def test_set_labels_resync_semantics():
    """Reading R12: pushing the labels the oracle already holds changes
    nothing (same trajectory as an untouched twin); moving one object marks
    both of its clusters moving, on top of the assignment's own changes, and
    the object loses its stored own score, so it is not filtered next time."""
    pin_set_labels()


def pin_set_labels(lib=None):
    w = CONFIGS["c1"].scaled(N=600, D=1500, k=12)
    c = generate(w.N, w.D, w.zipf_s, w.mu, w.sigma, w.lo, w.hi, 41)
    ini = init_ids(w.N, w.k, 41)
    a, b = Oracle(c, w.k, ini, icp=True, lib=lib), Oracle(c, w.k, ini, icp=True, lib=lib)
    for _ in range(3):
        a.assign(), b.assign()
        a.update(), b.update()
    a.assign(), b.assign()
    b.set_labels(b.labels())  # a no-op push
    assert np.array_equal(a.lam(), b.lam())
    for _ in range(3):
        ua, ub = a.update(), b.update()
        assert ua.objective == ub.objective
        aa, ab = a.assign(), b.assign()
        assert np.array_equal(a.labels(), b.labels()) and aa.filtered == ab.filtered
    # move one object of an invariant cluster to another invariant cluster
    lam, lab = b.lam(), b.labels()
    inv = np.nonzero(lam == 1)[0]
    assert len(inv) >= 2
    i = int(np.nonzero(lab == inv[0])[0][0])
    new = lab.copy()
    new[i] = inv[1]
    b.set_labels(new)
    lam2 = b.lam()
    assert lam2[inv[0]] == 0 and lam2[inv[1]] == 0
    assert np.all(lam2[lam == 0] == 0)  # the assignment's moving clusters stay moving
    b.update()
    b.assign()
    assert not b.scores()[2][i]  # own score dropped: not filtered
