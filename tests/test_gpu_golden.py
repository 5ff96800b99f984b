"""The CUDA path, through the C ABI, on the hand-worked runs under tests/golden/.

The same fixtures pin the FP64 oracle (tests/test_golden.py); here the GPU
must reproduce them in every ICP mode and posting precision: labels, change
counts and lambda exactly; similarity and posting counts and filtered objects
exactly for the unfiltered, SIVF and CBICP modes (for the relaxed filter the
GPU decides on error-bounded scores, so it may restrict fewer objects:
filtered <= and postings >= the hand-worked figures); objectives within 1e-6
relative; FP32 centroids and inverted-file values within 1e-5 relative of
the closed forms, with the exact sparsity pattern and posting order. With
CBICP (icp = 2) the file is unstructured (one part per list, ascending
centroid id), so there the ids of each list are compared as a set.
"""
from __future__ import annotations

import numpy as np
import pytest

from tests.golden_fixtures import FIXTURES, Golden
from tests.gpu_harness import CENTROID_RTOL, OBJECTIVE_RTOL, gpu_instance, rel

pytestmark = pytest.mark.gpu

CASES = [(n, m) for n in FIXTURES for m in Golden(n).modes]


def _check_close(got, want, what):
    got = np.asarray(got, dtype=np.float64)
    assert got.shape == want.shape, what
    assert np.all(np.abs(got - want) <= CENTROID_RTOL * np.abs(want)), f"{what}: {got} vs {want}"


@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp16"])
@pytest.mark.parametrize("name,mode", CASES, ids=[f"{n}-icp{m}" for n, m in CASES])
def test_cuda_path_reproduces_hand_worked_run(name, mode, precision):
    g = Golden(name)
    c = g.corpus()
    s = gpu_instance(c, g.k, g.seeds, precision=precision, icp=mode)
    try:
        for r in range(1, g.iterations + 1):
            what = f"{name} icp{mode} {precision} r={r}"
            changed = s.assign()
            st = s.stats()
            assert st["iter"] == r, what
            assert s.labels().tolist() == g[f"r{r}.labels"], what
            assert changed == st["changed"] == g[f"r{r}.changed"], what
            lam = g[f"r{r}.lambda"]
            assert s.lam().tolist() == lam, what
            assert st["n_moving"] == lam.count(0), what
            simcalc, postings, filtered = g[f"r{r}.icp{mode}"]
            if mode == 3:
                assert st["filtered"] <= filtered and st["postings"] >= postings, what
            else:
                assert (st["simcalc"], st["postings"], st["filtered"]) == (simcalc, postings, filtered), what
            if f"u{r}.objective" not in g:
                assert r == g.iterations and changed == 0, what
                break
            s.update()
            st = s.stats()
            assert rel(st["objective_assign"], g.num(f"r{r}.objective")) <= OBJECTIVE_RTOL, what
            assert rel(st["objective_update"], g.num(f"u{r}.objective")) <= OBJECTIVE_RTOL, what
            M = g.nums(f"u{r}.centroids")
            off, term, u = s.centroids()
            for j in range(g.k):
                sup = np.nonzero(M[j])[0]
                assert term[off[j]:off[j + 1]].tolist() == sup.tolist(), f"{what} centroid {j}"
                _check_close(u[off[j]:off[j + 1]], M[j, sup], f"{what} centroid {j}")
            if_off, mf0, cid, uu = s.inverted_file()
            want_cid, want_u = np.asarray(g[f"u{r}.if_cid"]), g.nums(f"u{r}.if_u")
            assert if_off.tolist() == g[f"u{r}.if_off"], what
            if mode == 2:
                for t in range(g.D):
                    a, b = if_off[t], if_off[t + 1]
                    assert cid[a:b].tolist() == sorted(want_cid[a:b].tolist()), f"{what} list {t}"
                    _check_close(uu[a:b], M[cid[a:b], t], f"{what} list {t}")
            else:
                assert mf0.tolist() == g[f"u{r}.if_mf0"], what
                assert cid.tolist() == want_cid.tolist(), what
                _check_close(uu, want_u, what)
    finally:
        s.close()
