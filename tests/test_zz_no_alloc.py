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


def _noalloc_inverted_file(g, torch):
    from paper_2103_16141_gb300 import sivf as S

    off_c, term_c, u_c = g.centroids()
    lam = g.lam()
    dev = torch.device("cuda", torch.cuda.current_device())
    coff = torch.from_numpy(off_c).to(dev)
    cterm = torch.from_numpy(term_c).to(dev)
    cval = torch.from_numpy(u_c).to(dev)
    lam_d = torch.from_numpy(lam).to(dev)
    n = int(off_c[-1])
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
