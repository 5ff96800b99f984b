"""CPU-side checks of the C ABI: the library builds for sm_103a, loads without
a GPU, and exports every function declared in include/sivf.h."""
from __future__ import annotations

import ctypes
import os
import re

from paper_2103_16141_gb300 import _build

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "sivf.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(sivf_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["sivf_init", "sivf_assign", "sivf_update", "sivf_run", "sivf_get_labels", "sivf_set_labels",
                     "sivf_get_centroids", "sivf_get_stats", "sivf_last_error", "sivf_destroy"]:
        assert required in names


def test_library_loads_and_exports_every_declared_symbol():
    path = _build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_null_context_is_rejected_without_a_gpu():
    lib = ctypes.CDLL(_build.build())
    lib.sivf_assign.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    lib.sivf_update.argtypes = [ctypes.c_void_p]
    lib.sivf_last_error.argtypes = [ctypes.c_void_p]
    lib.sivf_last_error.restype = ctypes.c_char_p
    lib.sivf_destroy.argtypes = [ctypes.c_void_p]
    assert lib.sivf_assign(None, None) == 1  # SIVF_ERR_INVALID_ARG
    assert lib.sivf_update(None) == 1
    assert lib.sivf_last_error(None)
    lib.sivf_destroy(None)


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.dirname(_build.__file__)
    for root, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(root, f)).read()
                assert "oracle" not in re.findall(r"import\s+(\w+)", text)
                assert "from oracle" not in text and "import oracle" not in text


def _struct_fields(name):
    """Member names, in order, of `typedef struct { ... } name;` in sivf.h."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    m = re.search(r"typedef struct\s*\{([^{}]*)\}\s*" + name + r"\s*;", text)
    assert m, name
    fields = []
    for decl in m.group(1).split(";"):
        decl = decl.strip()
        if decl:
            fields.append(re.findall(r"(\w+)\s*$", decl)[0])
    return fields


def test_binding_structs_match_the_header():
    """The ctypes mirrors of sivf_config, sivf_stats and sivf_instance_desc
    list the header's members in the header's order (a mismatch would shift
    every later member)."""
    from paper_2103_16141_gb300 import sivf as S
    for cname, cls in [("sivf_config", S.sivf_config), ("sivf_stats", S.sivf_stats),
                       ("sivf_instance_desc", S.sivf_instance_desc)]:
        assert [f for f, _ in cls._fields_] == _struct_fields(cname), cname


def test_binding_struct_sizes_match_the_compiler():
    """sizeof of each struct as gcc lays it out from the header equals the
    ctypes size."""
    import subprocess
    import tempfile
    from paper_2103_16141_gb300 import sivf as S
    src = ('#include <stdio.h>\n#include "sivf.h"\nint main(void){printf("%zu %zu %zu\\n", sizeof(sivf_config), '
           'sizeof(sivf_stats), sizeof(sivf_instance_desc));return 0;}\n')
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "s.c")
        exe = os.path.join(d, "s")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-I", os.path.dirname(HEADER), "-o", exe, c])
        sizes = [int(x) for x in subprocess.check_output([exe]).split()]
    assert sizes == [ctypes.sizeof(S.sivf_config), ctypes.sizeof(S.sivf_stats), ctypes.sizeof(S.sivf_instance_desc)]


def test_no_cpu_fallback_without_a_gpu():
    """Without a CUDA device the binding refuses to run (there is no CPU
    path): creating a context raises instead of computing anything."""
    import numpy as np
    import pytest
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2103_16141_gb300 import SIVF
    from tests.helpers import random_dense_corpus
    _, c = random_dense_corpus(20, 10, 0.5, seed=1)
    with pytest.raises(Exception):
        SIVF(c.row_ptr, c.idx, c.val, c.D, 2, np.array([0, 1], dtype=np.int32))


def test_icp_mode_names():
    from paper_2103_16141_gb300.sivf import icp_mode
    assert [icp_mode(x) for x in (False, True, 0, 1, 2, 3, "cbicp", "relaxed")] == [0, 1, 0, 1, 2, 3, 2, 3]


def test_init_rejects_bad_arguments_before_touching_the_device():
    """sivf_init and sivf_batch_init check sizes, pointers, configuration and
    seed ids on the host before any CUDA call: every rejection below returns
    its status and leaves *out NULL, with no GPU present."""
    import numpy as np
    from paper_2103_16141_gb300 import sivf as S
    lib = ctypes.CDLL(_build.build())
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
    lib.sivf_init.argtypes = [ctypes.POINTER(vp), vp, i64, i32, i32, vp, vp, vp, vp, vp]
    lib.sivf_batch_init.argtypes = [ctypes.POINTER(vp), vp, i32, vp, vp]
    INVALID, BAD_CSR = 1, 2

    row_ptr = np.array([0, 1, 2, 3, 4], dtype=np.int64)
    idx = np.zeros(4, dtype=np.int32)
    val = np.ones(4, dtype=np.float32)
    seeds = np.array([0, 1], dtype=np.int32)
    P = lambda a: a.ctypes.data  # noqa: E731

    def init(cfg=None, N=4, D=3, k=2, rp=P(row_ptr), ix=P(idx), vl=P(val), ini=P(seeds), out=True):
        h = vp(12345)
        st = lib.sivf_init(ctypes.byref(h) if out else None, ctypes.byref(cfg) if cfg else None,
                           N, D, k, rp, ix, vl, ini, None)
        if out:
            assert h.value is None, "out must be cleared on failure"
        return st

    def cfg(**kw):
        c = S.sivf_config()
        c.prec, c.icp = 0, 1
        for key, v in kw.items():
            setattr(c, key, v)
        return c

    assert init(out=False) == INVALID
    for kw in [dict(N=0), dict(D=0), dict(k=0), dict(k=5), dict(N=1 << 31), dict(D=(1 << 30) + 1),
               dict(rp=None), dict(ix=None), dict(vl=None), dict(ini=None)]:
        assert init(**kw) == INVALID, kw
    for kw in [dict(prec=3), dict(prec=-1), dict(icp=4), dict(icp=-1)]:
        assert init(cfg(**kw)) == INVALID, kw
    for bad in ([0, 0], [0, 4], [-1, 1]):
        assert init(ini=P(np.array(bad, dtype=np.int32))) == INVALID, bad
    # host inputs: the CSR header is read on the host first
    shifted = np.array([1, 2, 3, 4, 5], dtype=np.int64)
    assert init(cfg(inputs_on_host=1), rp=P(shifted)) == BAD_CSR

    def batch(descs, c=None, n=None):
        arr = (S.sivf_instance_desc * max(len(descs), 1))(*descs)
        h = vp(12345)
        st = lib.sivf_batch_init(ctypes.byref(h), ctypes.byref(c) if c else None,
                                 len(descs) if n is None else n, ctypes.addressof(arr), None)
        assert h.value is None
        return st

    def desc(N=4, D=3, k=2, ini=seeds):
        return S.sivf_instance_desc(N, D, k, P(row_ptr), P(idx), P(val), P(ini))

    assert batch([desc()], n=0) == INVALID
    assert batch([desc()], n=65537) == INVALID
    assert batch([desc()], c=cfg(inputs_on_host=1)) == INVALID
    assert batch([desc()], c=cfg(icp=5)) == INVALID
    assert batch([desc(), desc(k=5)]) == INVALID
    assert batch([desc(), desc(ini=np.array([1, 1], dtype=np.int32))]) == INVALID


def test_binding_checks_array_sizes_before_the_library_reads_them():
    """The library reads row_ptr[N] idx and val entries, k seed ids and N
    labels from the pointers it is given; the binding rejects shorter (or
    longer) arrays and a label buffer of the wrong kind before any call."""
    import numpy as np
    import pytest
    import torch
    from paper_2103_16141_gb300 import sivf as S

    rp = np.array([0, 2, 3], dtype=np.int64)
    S._check_csr_sizes(rp, np.zeros(3, np.int32), np.ones(3, np.float32))
    for ix, vl in [(2, 3), (3, 2), (4, 3)]:
        with pytest.raises(ValueError):
            S._check_csr_sizes(rp, np.zeros(ix, np.int32), np.ones(vl, np.float32))
    with pytest.raises(ValueError):
        S._check_csr_sizes(np.array([0], dtype=np.int64), np.zeros(0, np.int32), np.ones(0, np.float32))

    class Ctx:  # stands in for a live context; no call reaches the library
        N, k, ctx, device = 4, 2, None, torch.device("cuda", 0)

    with pytest.raises(ValueError):
        S.SIVF.set_labels(Ctx(), np.zeros(3, np.int32))
    with pytest.raises(ValueError):
        S.SIVF.reseed(Ctx(), [0])
    for out in (torch.zeros(4, dtype=torch.int32), torch.zeros(4, dtype=torch.int64), [0, 0, 0, 0]):
        with pytest.raises(ValueError):
            S.SIVF.labels_device(Ctx(), out=out)


def test_noalloc_rejects_sizes_beyond_its_limits_on_the_host():
    """The allocation-free build checks k, D, n_entries and the pointers on the
    host before any CUDA call (no GPU needed); the device arrays are never
    read (the pointers below are not even valid)."""
    from paper_2103_16141_gb300 import sivf as S
    lib = S.load()
    INVALID = S.SIVF_ERR_INVALID_ARG
    limits = dict(k=1 << 20, D=1 << 18, n=1 << 20)
    for k, D, n in [(limits["k"] + 1, 100, 10), (4, limits["D"] + 1, 10), (4, 100, limits["n"] + 1),
                    (0, 100, 10), (4, 0, 10), (4, 100, -1)]:
        assert lib.sivf_build_inverted_file_noalloc(k, D, n, 1, 1, 1, 1, 1, 1, 1, 1, None) == INVALID, (k, D, n)
    # NULL pointers
    assert lib.sivf_build_inverted_file_noalloc(4, 100, 10, None, 1, 1, 1, 1, 1, 1, 1, None) == INVALID
    assert lib.sivf_build_inverted_file_noalloc(4, 100, 10, 1, None, 1, 1, 1, 1, 1, 1, None) == INVALID
