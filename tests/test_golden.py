"""The FP64 oracle against the hand-worked runs stored under tests/golden/.

Each fixture is a run of the method worked by hand from its definitions
(Algorithm 1 loop; Algorithms 2, 4, 3 and the relaxed filter of Section 3 for
the assignment; Algorithm 5 for the update and the structured inverted file;
Section 6 for the similarity counts). The oracle must reproduce, in every ICP
mode, each assignment's labels, change count, lambda, objective, similarity
and posting counts and filtered objects, and each update's objective,
centroids (values and support) and inverted file (offsets, front lengths,
centroid ids, values).
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import Oracle
from tests.golden_fixtures import FIXTURES, Golden

TOL = 1e-14  # absolute; every value is O(1) and FP64 rounding differs only in order


def check_fixture(name: str, mode: int, lib=None) -> None:
    g = Golden(name)
    c = g.corpus()
    o = Oracle(c, g.k, g.seeds, icp=mode, lib=lib)
    for r in range(1, g.iterations + 1):
        a = o.assign()
        what = f"{name} icp{mode} r={r}"
        assert a.r == r, what
        assert o.labels().tolist() == g[f"r{r}.labels"], what
        assert a.changed == g[f"r{r}.changed"], what
        lam = g[f"r{r}.lambda"]
        assert o.lam().tolist() == lam, what
        assert a.n_moving == lam.count(0), what
        assert abs(a.objective - g.num(f"r{r}.objective")) <= TOL, what
        assert (a.simcalc, a.postings, a.filtered) == tuple(g[f"r{r}.icp{mode}"]), what
        best, second, filt = o.scores()
        if f"r{r}.best" in g:
            np.testing.assert_allclose(best, g.nums(f"r{r}.best"), rtol=0, atol=TOL, err_msg=what)
        if f"r{r}.second" in g:
            np.testing.assert_allclose(second, g.nums(f"r{r}.second"), rtol=0, atol=TOL, err_msg=what)
        if f"r{r}.filtered_icp{mode}" in g:
            assert filt.tolist() == g[f"r{r}.filtered_icp{mode}"], what
        if f"u{r}.objective" not in g:
            assert r == g.iterations and a.changed == 0, what
            break
        u = o.update()
        what = f"{name} icp{mode} update {r}"
        assert abs(u.objective - g.num(f"u{r}.objective")) <= TOL, what
        assert u.empty == (g[f"u{r}.empty"] if f"u{r}.empty" in g else 0), what
        M = g.nums(f"u{r}.centroids")
        np.testing.assert_allclose(o.dense_centroids(), M, rtol=0, atol=TOL, err_msg=what)
        off, term, _, _ = o.centroids()
        support = [sorted(term[off[j]:off[j + 1]].tolist()) for j in range(g.k)]
        assert support == [np.nonzero(M[j])[0].tolist() for j in range(g.k)], what
        if_off, mf0, cid, uu = o.inverted_file()
        assert if_off.tolist() == g[f"u{r}.if_off"], what
        assert mf0.tolist() == g[f"u{r}.if_mf0"], what
        assert cid.tolist() == g[f"u{r}.if_cid"], what
        np.testing.assert_allclose(uu, g.nums(f"u{r}.if_u"), rtol=0, atol=TOL, err_msg=what)
    # the Algorithm 1 loop stops at the same assignment
    hist = Oracle(c, g.k, g.seeds, icp=mode, lib=lib).run(10 * g.iterations)
    assert len(hist) == g.iterations and hist[-1][1] is None


def pin_golden(lib=None) -> None:
    for name in FIXTURES:
        for mode in Golden(name).modes:
            check_fixture(name, mode, lib)


CASES = [(n, m) for n in FIXTURES for m in Golden(n).modes]


@pytest.mark.parametrize("name,mode", CASES, ids=[f"{n}-icp{m}" for n, m in CASES])
def test_oracle_reproduces_hand_worked_run(name, mode):
    check_fixture(name, mode)


def test_fixtures_present():
    assert {"hand_icp_k4", "hand_ties_empty_k3", "hand_two_blocks_k2"} <= set(FIXTURES)


def test_fixture_documents_are_unit_or_empty_rows():
    for name in FIXTURES:
        n = np.linalg.norm(Golden(name).dense().astype(np.float64), axis=1)
        assert np.all((n == 0.0) | (np.abs(n - 1.0) <= 1e-7)), name
