"""The allocation-free inverted-file build (sivf_build_inverted_file_noalloc)
gives exactly the inverted file that the regular update step builds.

Callers that may not allocate device memory (engine plugins, services with a
fixed device-memory budget) use this entry point; its scratch is a static
device array shared by every call. The test feeds it the centroids and lambda
of a live context, twice in a row on different states, and compares with the
context's own inverted file (sivf_get_inverted_file). The comparison is
bit-exact, as for every integer and copied value in the other GPU tests.

This file is named to be collected last, so that a run stopping at its first
failure has already run every other test.
"""
from __future__ import annotations

import numpy as np
import pytest

from synth import CONFIGS
from tests.gpu_harness import corpus_for, gpu_instance

pytestmark = pytest.mark.gpu


def _noalloc_inverted_file(g, torch, off_c=None, term_c=None):
    from paper_2103_16141_gb300 import sivf as S

    off0, term0, u_c = g.centroids()
    off_c = off0 if off_c is None else off_c
    term_c = term0 if term_c is None else term_c
    lam = g.lam()
    dev = torch.device("cuda", torch.cuda.current_device())
    coff = torch.from_numpy(off_c).to(dev)
    cterm = torch.from_numpy(term_c).to(dev)
    cval = torch.from_numpy(u_c).to(dev)
    lam_d = torch.from_numpy(lam).to(dev)
    n = len(term_c)
    if_off = torch.full((g.D + 1,), -1, dtype=torch.int64, device=dev)
    mf0 = torch.full((g.D,), -1, dtype=torch.int32, device=dev)
    cid = torch.full((max(n, 1),), -1, dtype=torch.int32, device=dev)
    uu = torch.full((max(n, 1),), -1.0, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    S.sivf_build_inverted_file_noalloc(g.k, g.D, n, coff.data_ptr(), cterm.data_ptr(), cval.data_ptr(),
                                       lam_d.data_ptr(), if_off.data_ptr(), mf0.data_ptr(), cid.data_ptr(),
                                       uu.data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize()
    return if_off.cpu().numpy(), mf0.cpu().numpy(), cid.cpu().numpy()[:n], uu.cpu().numpy()[:n]


def test_noalloc_inverted_file_matches_update_step_twice():
    torch = pytest.importorskip("torch")
    w = CONFIGS["c2"].scaled(N=6_000, D=8_000, k=60)
    c, ini = corpus_for(w, seed=21)
    g = gpu_instance(c, w.k, ini)
    try:
        compared = 0
        for it in range(6):
            g.assign()
            g.update()
            if it < 3:
                continue  # compare on two consecutive later states (moving and invariant parts present)
            ref = g.inverted_file()
            got = _noalloc_inverted_file(g, torch)
            for name, a, b in zip(("off", "mf0", "cid", "u"), got, ref):
                assert np.array_equal(a, b), f"call {compared + 1}: {name} differs"
            compared += 1
            if compared == 2:
                break
        assert compared == 2
    finally:
        g.close()


def test_noalloc_rejects_sizes_beyond_its_limits():
    from paper_2103_16141_gb300 import sivf as S

    lib = S.load()
    too_many = (1 << 20) + 1
    st = lib.sivf_build_inverted_file_noalloc(4, 100, too_many, 1, 1, 1, 1, 1, 1, 1, 1, None)
    assert st == S.SIVF_ERR_INVALID_ARG
    st = lib.sivf_build_inverted_file_noalloc(4, (1 << 18) + 1, 10, 1, 1, 1, 1, 1, 1, 1, 1, None)
    assert st == S.SIVF_ERR_INVALID_ARG


def test_noalloc_rejects_malformed_centroids_on_the_device_then_still_builds():
    """The offsets and terms are device data that the host cannot see: the
    entry point checks them on the device (its own bounds checks, every
    access in bounds) and returns SIVF_ERR_INVALID_ARG for offsets that do not
    end at n_entries, offsets that decrease, or a term >= D. A valid call made
    after those failures still gives the update step's inverted file."""
    torch = pytest.importorskip("torch")
    from paper_2103_16141_gb300 import sivf as S

    w = CONFIGS["c2"].scaled(N=3_000, D=5_000, k=40)
    c, ini = corpus_for(w, seed=5)
    g = gpu_instance(c, w.k, ini)
    try:
        for _ in range(3):
            g.assign()
            g.update()
        off, term, _ = g.centroids()
        n = int(off[-1])
        long_end = off.copy()
        long_end[-1] = n + 3  # coff[k] != n_entries
        decreasing = off.copy()
        decreasing[w.k // 2] = decreasing[w.k // 2 + 1] + 1  # still ends at n_entries
        bad_term = term.copy()
        bad_term[n // 2] = w.D  # outside [0, D)
        for what, o, t in (("coff[k] != n_entries", long_end, term), ("decreasing coff", decreasing, term),
                           ("term >= D", off, bad_term)):
            with pytest.raises(S.SivfError) as ex:
                _noalloc_inverted_file(g, torch, off_c=o, term_c=t)
            assert ex.value.status == S.SIVF_ERR_INVALID_ARG, what
        ref = g.inverted_file()
        got = _noalloc_inverted_file(g, torch)
        for name, a, b in zip(("off", "mf0", "cid", "u"), got, ref):
            assert np.array_equal(a, b), f"after the rejected calls: {name} differs"
    finally:
        g.close()
