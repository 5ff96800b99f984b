"""Failure handling of the C ABI on the GPU, with bad inputs made on the host.

Every case below is caught by a check of the library itself (on the host, or
a device-side check that reads nothing through the bad value and records a
status word), so no kernel ever reads out of bounds:
  - a malformed CSR is rejected at init by the validation kernel
    (SIVF_ERR_BAD_CSR): terms out of order or out of range, values <= 0, a
    row norm off 1 by more than 1e-4;
  - a memory cap below what the context needs gives SIVF_ERR_OOM;
  - in checked mode, a borrowed CSR corrupted after init is caught by the
    assignment kernel's own checks: SIVF_ERR_STATE, the context stays latched;
  - sivf_reseed forgets the previous run's objective.
"""
from __future__ import annotations

import numpy as np
import pytest

from synth import CONFIGS
from tests.gpu_harness import corpus_for, gpu_instance

pytestmark = pytest.mark.gpu


def _small():
    w = CONFIGS["c1"].scaled(N=400, D=1_500, k=12)
    return w, *corpus_for(w, seed=3)


def _row_with(c, n_min):
    lens = np.diff(c.row_ptr)
    return int(np.nonzero(lens >= n_min)[0][0])


@pytest.mark.parametrize("flaw", ["unsorted", "term_eq_D", "term_negative", "zero_value", "negative_value",
                                  "norm_off"])
def test_malformed_csr_is_rejected_at_init(flaw):
    from paper_2103_16141_gb300 import sivf as S
    w, c, ini = _small()
    idx, val = c.idx.copy(), c.val.copy()
    i = _row_with(c, 3)
    b = int(c.row_ptr[i])
    if flaw == "unsorted":
        idx[b], idx[b + 1] = idx[b + 1], idx[b]
    elif flaw == "term_eq_D":
        idx[int(c.row_ptr[i + 1]) - 1] = w.D
    elif flaw == "term_negative":
        idx[b] = -1
    elif flaw == "zero_value":
        val[b] = 0.0
    elif flaw == "negative_value":
        val[b] = -val[b]
    elif flaw == "norm_off":
        e = int(c.row_ptr[i + 1])
        val[b:e] *= np.float32(1.001)  # norm 1.001: off by 1e-3 > 1e-4
    with pytest.raises(S.SivfError) as ex:
        S.SIVF(c.row_ptr, idx, val, w.D, w.k, ini)
    assert ex.value.status == S.SIVF_ERR_BAD_CSR, flaw


def test_norm_within_tolerance_is_accepted():
    """A row norm off by less than 1e-4 is not a malformed row."""
    from paper_2103_16141_gb300 import sivf as S
    w, c, ini = _small()
    val = c.val.copy()
    i = _row_with(c, 3)
    val[int(c.row_ptr[i]):int(c.row_ptr[i + 1])] *= np.float32(1.00002)
    g = S.SIVF(c.row_ptr, c.idx, val, w.D, w.k, ini)
    g.close()


def test_malformed_batch_instance_is_rejected():
    from paper_2103_16141_gb300 import SIVFBatch, sivf as S
    w, c, ini = _small()
    bad = type(c)(N=c.N, D=c.D, row_ptr=c.row_ptr, idx=c.idx.copy(), val=c.val)
    bad.idx[5] = w.D + 3
    with pytest.raises(S.SivfError) as ex:
        SIVFBatch([c, bad], [w.k, w.k], [ini, ini])
    assert ex.value.status == S.SIVF_ERR_BAD_CSR


def test_memory_cap_gives_oom():
    from paper_2103_16141_gb300 import sivf as S
    w, c, ini = _small()
    with pytest.raises(S.SivfError) as ex:
        S.SIVF(c.row_ptr, c.idx, c.val, w.D, w.k, ini, mem_cap_bytes=1 << 16)
    assert ex.value.status == S.SIVF_ERR_OOM
    # a cap that holds everything (the sort-form update needs no accumulator)
    g = S.SIVF(c.row_ptr, c.idx, c.val, w.D, w.k, ini, mem_cap_bytes=1 << 30)
    try:
        g.run(5)
    finally:
        g.close()


@pytest.mark.parametrize("corrupt", ["term", "row_ptr"])
def test_checked_mode_latches_on_a_csr_changed_after_init(corrupt):
    """The CSR is borrowed: a caller that changes it after sivf_init breaks the
    contract. In checked mode the assignment kernel checks offsets and terms
    before using them, so the bad value is never used as an index; the call
    returns SIVF_ERR_STATE and every later call too (latched)."""
    from paper_2103_16141_gb300 import sivf as S
    w, c, ini = _small()
    g = gpu_instance(c, w.k, ini, checked=True)
    try:
        for _ in range(2):
            g.assign()
            g.update()
        if corrupt == "term":
            g.idx[int(c.row_ptr[7])] = w.D + 7
        else:
            g.row_ptr[9] = int(c.row_ptr[-1]) + 100  # row 8 ends past nnz, row 9 ends before it starts
        with pytest.raises(S.SivfError) as ex:
            g.assign()
        assert ex.value.status == S.SIVF_ERR_STATE
        assert "device-side check" in g.last_error()
        for call in (g.update, g.assign, lambda: g.run(3), g.labels):
            with pytest.raises(S.SivfError) as ex:
                call()
            assert ex.value.status == S.SIVF_ERR_STATE
    finally:
        g.close()


def test_checked_mode_gives_the_unchecked_results():
    w, c, ini = _small()
    a = gpu_instance(c, w.k, ini, checked=True, use_graph=True)
    b = gpu_instance(c, w.k, ini, use_graph=True)
    try:
        ia, oa = a.run(30)
        ib, ob = b.run(30)
        assert (ia, oa) == (ib, ob)
        assert np.array_equal(a.labels(), b.labels())
        assert a.stats()["graph_iters"] == 0  # checked contexts step from the host
    finally:
        a.close()
        b.close()


def test_reseed_forgets_the_previous_objective():
    w, c, ini = _small()
    g = gpu_instance(c, w.k, ini)
    try:
        it, obj = g.run(6)
        assert it > 0 and obj > 0
        g.reseed(ini)
        it0, obj0 = g.run(0)
        assert it0 == 0 and obj0 == 0.0
        st = g.stats()
        assert st["objective_update"] == 0.0 and st["objective_assign"] == 0.0
        # and a fresh run from the same seeds reproduces the first one
        assert g.run(6) == (it, obj)
    finally:
        g.close()
