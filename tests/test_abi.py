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
