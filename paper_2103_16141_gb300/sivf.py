"""Python binding of libsivf.so (include/sivf.h): argument marshalling only.

Every step of the method runs in the CUDA library. PyTorch supplies device
memory and the stream. There is no CPU fallback: loading fails loudly when the
library is missing or cannot be loaded.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import _build

SIVF_OK, SIVF_ERR_INVALID_ARG, SIVF_ERR_BAD_CSR, SIVF_ERR_OOM, SIVF_ERR_CUDA, SIVF_ERR_TIMEOUT, SIVF_ERR_STATE = range(7)
STATUS_NAMES = ["SIVF_OK", "SIVF_ERR_INVALID_ARG", "SIVF_ERR_BAD_CSR", "SIVF_ERR_OOM", "SIVF_ERR_CUDA",
                "SIVF_ERR_TIMEOUT", "SIVF_ERR_STATE"]
PRECISIONS = {"fp32": 0, "bf16": 1, "fp16": 2}
SCORE_BUFFERS = {"auto": 0, "shared": 1, "global": 2}
UPDATE_MODES = {"auto": 0, "dense": 1, "sort": 2}


def icp_mode(icp) -> int:
    """False/0: unfiltered (Algorithm 2); True/1: SIVF (Algorithm 4);
    2 or "cbicp": IVF-CBICP (Algorithm 3); 3 or "relaxed": SIVF with the
    relaxed (own-similarity) filter."""
    if icp == "cbicp" or (not isinstance(icp, bool) and icp == 2):
        return 2
    if icp == "relaxed" or (not isinstance(icp, bool) and icp == 3):
        return 3
    return int(bool(icp))


class sivf_config(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int), ("icp", ctypes.c_int), ("threads", ctypes.c_int),
                ("ctas_per_sm", ctypes.c_int), ("mem_cap_bytes", ctypes.c_int64), ("use_graph", ctypes.c_int),
                ("autotune", ctypes.c_int), ("score_buffer", ctypes.c_int), ("update_mode", ctypes.c_int),
                ("inputs_on_host", ctypes.c_int), ("checked", ctypes.c_int),
                ("dense_max_bytes", ctypes.c_int64), ("dense_min_fraction", ctypes.c_float),
                ("light_max_moving", ctypes.c_int), ("dense_all", ctypes.c_int)]


class sivf_stats(ctypes.Structure):
    _fields_ = [("iter", ctypes.c_int32), ("changed", ctypes.c_int64), ("n_moving", ctypes.c_int64),
                ("n_moving_prev", ctypes.c_int64), ("filtered", ctypes.c_int64), ("simcalc", ctypes.c_int64),
                ("postings", ctypes.c_int64), ("rescored", ctypes.c_int64), ("rescore_cands", ctypes.c_int64),
                ("centroid_nnz", ctypes.c_int64), ("moved_nnz", ctypes.c_int64),
                ("objective_assign", ctypes.c_double), ("objective_update", ctypes.c_double),
                ("ms_assign", ctypes.c_double), ("ms_update", ctypes.c_double), ("launches", ctypes.c_int64),
                ("graph_iters", ctypes.c_int64), ("assign_threads", ctypes.c_int32),
                ("assign_global", ctypes.c_int32), ("update_dense", ctypes.c_int32),
                ("dense_entries", ctypes.c_int64), ("dense_postings", ctypes.c_int64),
                ("dense_terms", ctypes.c_int64), ("dense_row_entries", ctypes.c_int64),
                ("light_objects", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class sivf_instance_desc(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("D", ctypes.c_int32), ("k", ctypes.c_int32), ("row_ptr", ctypes.c_void_p),
                ("idx", ctypes.c_void_p), ("val", ctypes.c_void_p), ("init_ids", ctypes.c_void_p)]


class SivfError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libsivf.so (building it with nvcc if absent). Raises if it cannot."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing:
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"SIVF CUDA library not found at {path}; build it with __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        p, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        st = ctypes.c_int
        lib.sivf_init.argtypes = [ctypes.POINTER(p), ctypes.POINTER(sivf_config), i64, i32, i32, p, p, p, p, p]
        lib.sivf_init.restype = st
        lib.sivf_reseed.argtypes = [p, p]
        lib.sivf_reseed.restype = st
        lib.sivf_assign.argtypes = [p, ctypes.POINTER(i64)]
        lib.sivf_assign.restype = st
        lib.sivf_update.argtypes = [p]
        lib.sivf_update.restype = st
        lib.sivf_run.argtypes = [p, i32, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_double)]
        lib.sivf_run.restype = st
        lib.sivf_get_labels.argtypes = [p, p, ctypes.c_int]
        lib.sivf_get_labels.restype = st
        lib.sivf_set_labels.argtypes = [p, p, ctypes.c_int]
        lib.sivf_set_labels.restype = st
        lib.sivf_get_centroids.argtypes = [p, p, p, p, i64, ctypes.POINTER(i64)]
        lib.sivf_get_centroids.restype = st
        lib.sivf_get_inverted_file.argtypes = [p, p, p, p, p, i64, ctypes.POINTER(i64)]
        lib.sivf_get_inverted_file.restype = st
        lib.sivf_get_lambda.argtypes = [p, p]
        lib.sivf_get_lambda.restype = st
        lib.sivf_get_stats.argtypes = [p, ctypes.POINTER(sivf_stats)]
        lib.sivf_get_stats.restype = st
        lib.sivf_last_error.argtypes = [p]
        lib.sivf_last_error.restype = ctypes.c_char_p
        lib.sivf_destroy.argtypes = [p]
        lib.sivf_destroy.restype = None
        lib.sivf_batch_init.argtypes = [ctypes.POINTER(p), ctypes.POINTER(sivf_config), i32,
                                        ctypes.POINTER(sivf_instance_desc), p]
        lib.sivf_batch_init.restype = st
        lib.sivf_batch_run.argtypes = [p, i32, p, p]
        lib.sivf_batch_run.restype = st
        lib.sivf_batch_get_labels.argtypes = [p, i32, p]
        lib.sivf_batch_get_labels.restype = st
        lib.sivf_batch_instance_stats.argtypes = [p, i32, ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_double),
                                                  ctypes.POINTER(ctypes.c_double)]
        lib.sivf_batch_instance_stats.restype = st
        lib.sivf_build_inverted_file_noalloc.argtypes = [i32, i32, i64, p, p, p, p, p, p, p, p, p]
        lib.sivf_build_inverted_file_noalloc.restype = st
        lib.sivf_measure_read_bandwidth.argtypes = [p, i64, i32, p, ctypes.POINTER(ctypes.c_double),
                                                    ctypes.POINTER(ctypes.c_double)]
        lib.sivf_measure_read_bandwidth.restype = st
        _lib = lib
        return lib


def _check(lib, ctx, status: int):
    if status != SIVF_OK:
        msg = lib.sivf_last_error(ctx) if ctx else b""
        raise SivfError(status, (msg or b"").decode(errors="replace"))


# ---- thin wrappers with the C names (pointers are ints) ----

def sivf_init(cfg: sivf_config, N: int, D: int, k: int, row_ptr: int, idx: int, val: int, init_ids: int,
              stream: int) -> int:
    lib = load()
    ctx = ctypes.c_void_p()
    st = lib.sivf_init(ctypes.byref(ctx), ctypes.byref(cfg), N, D, k, row_ptr, idx, val, init_ids, stream)
    _check(lib, None, st)
    return ctx.value


def sivf_reseed(ctx: int, init_ids: int) -> None:
    lib = load()
    _check(lib, ctx, lib.sivf_reseed(ctx, init_ids))


def sivf_assign(ctx: int) -> int:
    lib = load()
    n = ctypes.c_int64(0)
    _check(lib, ctx, lib.sivf_assign(ctx, ctypes.byref(n)))
    return n.value


def sivf_update(ctx: int) -> None:
    lib = load()
    _check(lib, ctx, lib.sivf_update(ctx))


def sivf_run(ctx: int, max_iter: int):
    lib = load()
    it = ctypes.c_int32(0)
    obj = ctypes.c_double(0.0)
    _check(lib, ctx, lib.sivf_run(ctx, max_iter, ctypes.byref(it), ctypes.byref(obj)))
    return it.value, obj.value


def sivf_get_labels(ctx: int, dst: int, dst_is_device: bool) -> None:
    lib = load()
    _check(lib, ctx, lib.sivf_get_labels(ctx, dst, int(dst_is_device)))


def sivf_set_labels(ctx: int, src: int, src_is_device: bool) -> None:
    lib = load()
    _check(lib, ctx, lib.sivf_set_labels(ctx, src, int(src_is_device)))


def sivf_get_stats(ctx: int) -> sivf_stats:
    lib = load()
    s = sivf_stats()
    _check(lib, ctx, lib.sivf_get_stats(ctx, ctypes.byref(s)))
    return s


def sivf_build_inverted_file_noalloc(k: int, D: int, n_entries: int, coff: int, cterm: int, cval: int, lam: int,
                                     if_off: int, if_mf0: int, if_cid: int, if_u: int, stream: int) -> None:
    """Allocation-free inverted-file build (device pointers as ints; see
    include/sivf.h for who needs it and its size limits)."""
    lib = load()
    _check(lib, None, lib.sivf_build_inverted_file_noalloc(k, D, n_entries, coff, cterm, cval, lam, if_off, if_mf0,
                                                           if_cid, if_u, stream))


def sivf_measure_read_bandwidth(buf: int, nbytes: int, passes: int, stream: int):
    """(GB/s, ms) of `passes` streaming reads of a 16-byte-aligned device
    buffer (L2 -> SM when it fits in L2). See include/sivf.h."""
    lib = load()
    gbs, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(lib, None, lib.sivf_measure_read_bandwidth(buf, nbytes, passes, stream, ctypes.byref(gbs),
                                                      ctypes.byref(ms)))
    return gbs.value, ms.value


def sivf_destroy(ctx: int) -> None:
    if ctx:
        load().sivf_destroy(ctx)


def _check_csr_sizes(row_ptr, idx, val) -> None:
    """The library reads row_ptr[N] and then that many idx and val entries:
    the arrays must hold them (a short array would be read past its end)."""
    n = len(row_ptr)
    if n < 2:
        raise ValueError("row_ptr must hold N + 1 >= 2 offsets")
    nnz = int(row_ptr[n - 1])
    if len(idx) != nnz or len(val) != nnz:
        raise ValueError(f"idx and val must hold row_ptr[N] = {nnz} entries (got {len(idx)}, {len(val)})")


class SIVF:
    """One clustering instance on the current CUDA device.

    row_ptr / idx / val are torch tensors (int64 / int32 / float32) on the
    device, or numpy arrays that are copied to the device. The object keeps
    references to the device tensors for as long as the context lives, as the
    library borrows them.

    inputs_on_host=True passes HOST arrays (numpy, or CPU tensors, pinned for
    an asynchronous copy) straight to sivf_init, which copies them into device
    buffers of its own.
    """

    def __init__(self, row_ptr, idx, val, D: int, k: int, init_ids, precision: str = "fp32", icp=True,
                 threads: int = 0, ctas_per_sm: int = 0, mem_cap_bytes: int = 0, stream=None, use_graph: bool = False,
                 autotune: bool = False, score_buffer: str = "auto", inputs_on_host: bool = False,
                 update_mode: str = "auto", checked: bool = False, dense_max_bytes: int = 0,
                 dense_min_fraction: float = 0.0, light_max_moving: int = 0, dense_all: bool = False):
        import numpy as np
        import torch

        dev = torch.device("cuda", torch.cuda.current_device())

        def to_dev(a, dtype):
            if isinstance(a, torch.Tensor):
                return a.to(device=dev, dtype=dtype).contiguous()
            return torch.from_numpy(np.ascontiguousarray(a)).to(device=dev, dtype=dtype)

        def host(a, dtype):
            if isinstance(a, torch.Tensor):
                if a.is_cuda or a.dtype != dtype or not a.is_contiguous():
                    raise ValueError("inputs_on_host expects contiguous CPU tensors of the CSR dtypes")
                return a, a.data_ptr()
            a = np.ascontiguousarray(a, dtype={torch.int64: np.int64, torch.int32: np.int32,
                                               torch.float32: np.float32}[dtype])
            return a, a.ctypes.data

        if inputs_on_host:
            # nothing is borrowed: the library copies the host arrays at init
            (rp, rp_p), (ix, ix_p), (vl, vl_p) = (host(row_ptr, torch.int64), host(idx, torch.int32),
                                                  host(val, torch.float32))
            _check_csr_sizes(rp, ix, vl)
            self.row_ptr = self.idx = self.val = None
            self.N = int(len(rp) - 1)
        else:
            self.row_ptr = to_dev(row_ptr, torch.int64)
            self.idx = to_dev(idx, torch.int32)
            self.val = to_dev(val, torch.float32)
            _check_csr_sizes(self.row_ptr, self.idx, self.val)
            rp_p, ix_p, vl_p = self.row_ptr.data_ptr(), self.idx.data_ptr(), self.val.data_ptr()
            self.N = int(self.row_ptr.numel() - 1)
        self.D, self.k = int(D), int(k)
        self.device = dev
        ini = np.ascontiguousarray(np.asarray(init_ids, dtype=np.int32))
        if ini.shape != (self.k,):  # the library reads k ids
            raise ValueError(f"init_ids must hold k = {self.k} ids")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        cfg = sivf_config(PRECISIONS[precision], icp_mode(icp), int(threads), int(ctas_per_sm), int(mem_cap_bytes),
                          int(bool(use_graph)), int(bool(autotune)), SCORE_BUFFERS[score_buffer],
                          UPDATE_MODES[update_mode], int(bool(inputs_on_host)), int(bool(checked)),
                          int(dense_max_bytes), float(dense_min_fraction), int(light_max_moving),
                          int(bool(dense_all)))
        self.ctx = sivf_init(cfg, self.N, self.D, self.k, rp_p, ix_p, vl_p, ini.ctypes.data, self.stream.cuda_stream)

    def close(self):
        if getattr(self, "ctx", None):
            sivf_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reseed(self, init_ids) -> None:
        import numpy as np
        ini = np.ascontiguousarray(np.asarray(init_ids, dtype=np.int32))
        if ini.shape != (self.k,):  # the library reads k ids
            raise ValueError(f"init_ids must hold k = {self.k} ids")
        sivf_reseed(self.ctx, ini.ctypes.data)

    def assign(self) -> int:
        return sivf_assign(self.ctx)

    def update(self) -> None:
        sivf_update(self.ctx)

    def run(self, max_iter: int):
        return sivf_run(self.ctx, max_iter)

    def stats(self) -> dict:
        return sivf_get_stats(self.ctx).as_dict()

    def last_error(self) -> str:
        return (load().sivf_last_error(self.ctx) or b"").decode(errors="replace")

    def labels(self):
        import numpy as np
        out = np.empty(self.N, dtype=np.int32)
        sivf_get_labels(self.ctx, out.ctypes.data, False)
        return out

    def labels_device(self, out=None):
        """Labels into a device tensor (int32[N] on the context's device; a new
        one if out is None). The library writes N int32 values, so out is
        checked first."""
        import torch
        if out is None:
            out = torch.empty(self.N, dtype=torch.int32, device=self.device)
        elif (not isinstance(out, torch.Tensor) or out.device != self.device or out.dtype != torch.int32
              or not out.is_contiguous() or out.numel() != self.N):
            raise ValueError(f"out must be a contiguous int32 tensor of {self.N} elements on {self.device}")
        sivf_get_labels(self.ctx, out.data_ptr(), True)
        return out

    def set_labels(self, labels) -> None:
        import numpy as np
        import torch
        # the library reads N labels from the pointer it is given
        if isinstance(labels, torch.Tensor) and labels.is_cuda:
            t = labels.to(device=self.device, dtype=torch.int32).contiguous()
            if t.shape != (self.N,):
                raise ValueError(f"labels must hold N = {self.N} entries")
            sivf_set_labels(self.ctx, t.data_ptr(), True)
        else:
            a = np.ascontiguousarray(np.asarray(labels, dtype=np.int32))
            if a.shape != (self.N,):
                raise ValueError(f"labels must hold N = {self.N} entries")
            sivf_set_labels(self.ctx, a.ctypes.data, False)

    def lam(self):
        import numpy as np
        lib = load()
        out = np.empty(self.k, dtype=np.uint8)
        _check(lib, self.ctx, lib.sivf_get_lambda(self.ctx, out.ctypes.data))
        return out

    def centroids(self):
        """(off[k+1], term[nnz], u[nnz] fp32), cluster-major master copy."""
        import numpy as np
        lib = load()
        off = np.empty(self.k + 1, dtype=np.int64)
        n = ctypes.c_int64(0)
        st = lib.sivf_get_centroids(self.ctx, off.ctypes.data, None, None, 0, ctypes.byref(n))
        if st not in (SIVF_OK, SIVF_ERR_INVALID_ARG):
            _check(lib, self.ctx, st)
        term = np.empty(max(n.value, 1), dtype=np.int32)
        u = np.empty(max(n.value, 1), dtype=np.float32)
        _check(lib, self.ctx, lib.sivf_get_centroids(self.ctx, off.ctypes.data, term.ctypes.data, u.ctypes.data,
                                                     len(term), ctypes.byref(n)))
        return off, term[:n.value], u[:n.value]

    def inverted_file(self):
        """(off[D+1], mf0[D], cid[nnz], u[nnz] fp32) of the structured inverted file."""
        import numpy as np
        lib = load()
        off = np.empty(self.D + 1, dtype=np.int64)
        mf0 = np.empty(self.D, dtype=np.int32)
        n = ctypes.c_int64(0)
        st = lib.sivf_get_inverted_file(self.ctx, off.ctypes.data, mf0.ctypes.data, None, None, 0, ctypes.byref(n))
        if st not in (SIVF_OK, SIVF_ERR_INVALID_ARG):
            _check(lib, self.ctx, st)
        cid = np.empty(max(n.value, 1), dtype=np.int32)
        u = np.empty(max(n.value, 1), dtype=np.float32)
        _check(lib, self.ctx, lib.sivf_get_inverted_file(self.ctx, off.ctypes.data, mf0.ctypes.data,
                                                         cid.ctypes.data, u.ctypes.data, len(cid), ctypes.byref(n)))
        return off, mf0, cid[:n.value], u[:n.value]


def sivf_batch_init(cfg: sivf_config, descs) -> int:
    lib = load()
    arr = (sivf_instance_desc * len(descs))(*descs)
    ctx = ctypes.c_void_p()
    _check(lib, None, lib.sivf_batch_init(ctypes.byref(ctx), ctypes.byref(cfg), len(descs), arr,
                                          _current_stream()))
    return ctx.value


def _current_stream() -> int:
    import torch
    return torch.cuda.current_stream().cuda_stream


class SIVFBatch:
    """Many independent instances in one context (sivf_batch_init).

    corpora: list of objects with row_ptr, idx, val (numpy or torch), D;
    ks: clusters per instance; init_ids: per-instance local seed ids.
    """

    def __init__(self, corpora, ks, init_ids, precision: str = "fp32", icp=True, threads: int = 0,
                 ctas_per_sm: int = 0, use_graph: bool = False, autotune: bool = False, score_buffer: str = "auto",
                 update_mode: str = "auto", dense_max_bytes: int = 0, dense_min_fraction: float = 0.0,
                 light_max_moving: int = 0):
        import numpy as np
        import torch

        dev = torch.device("cuda", torch.cuda.current_device())
        corpora, ks, init_ids = list(corpora), list(ks), list(init_ids)
        if not (len(corpora) == len(ks) == len(init_ids)):
            raise ValueError("corpora, ks and init_ids must have one entry per instance")
        self._keep = []
        descs = []
        for c, k, ini in zip(corpora, ks, init_ids):
            rp = torch.as_tensor(np.ascontiguousarray(c.row_ptr), dtype=torch.int64).to(dev)
            ix = torch.as_tensor(np.ascontiguousarray(c.idx), dtype=torch.int32).to(dev)
            vl = torch.as_tensor(np.ascontiguousarray(c.val), dtype=torch.float32).to(dev)
            _check_csr_sizes(rp, ix, vl)
            ii = np.ascontiguousarray(np.asarray(ini, dtype=np.int32))
            if ii.shape != (int(k),):  # the library reads k ids
                raise ValueError(f"init_ids of an instance must hold its k = {int(k)} ids")
            self._keep.append((rp, ix, vl, ii))
            descs.append(sivf_instance_desc(int(rp.numel() - 1), int(c.D), int(k), rp.data_ptr(), ix.data_ptr(),
                                            vl.data_ptr(), ii.ctypes.data))
        self.n_inst = len(descs)
        self.Ns = [d.N for d in descs]
        self.ks = [int(k) for k in ks]
        cfg = sivf_config(PRECISIONS[precision], icp_mode(icp), int(threads), int(ctas_per_sm), 0,
                          int(bool(use_graph)), int(bool(autotune)), SCORE_BUFFERS[score_buffer],
                          UPDATE_MODES[update_mode], 0, 0, int(dense_max_bytes), float(dense_min_fraction),
                          int(light_max_moving))
        self.ctx = sivf_batch_init(cfg, descs)
        self._keep = None  # the library copied the corpora

    def close(self):
        if getattr(self, "ctx", None):
            sivf_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def assign(self) -> int:
        return sivf_assign(self.ctx)

    def update(self) -> None:
        sivf_update(self.ctx)

    def run(self, max_iter: int):
        import numpy as np
        lib = load()
        it = np.zeros(self.n_inst, dtype=np.int32)
        obj = np.zeros(self.n_inst, dtype=np.float64)
        _check(lib, self.ctx, lib.sivf_batch_run(self.ctx, max_iter, it.ctypes.data, obj.ctypes.data))
        return it, obj

    def labels(self, inst: int):
        import numpy as np
        lib = load()
        out = np.empty(self.Ns[inst], dtype=np.int32)
        _check(lib, self.ctx, lib.sivf_batch_get_labels(self.ctx, inst, out.ctypes.data))
        return out

    def instance_stats(self, inst: int) -> dict:
        lib = load()
        ch = ctypes.c_int64(0)
        ja, ju = ctypes.c_double(0), ctypes.c_double(0)
        _check(lib, self.ctx, lib.sivf_batch_instance_stats(self.ctx, inst, ctypes.byref(ch), ctypes.byref(ja),
                                                            ctypes.byref(ju)))
        return {"changed": ch.value, "objective_assign": ja.value, "objective_update": ju.value}

    def stats(self) -> dict:
        return sivf_get_stats(self.ctx).as_dict()

    def last_error(self) -> str:
        return (load().sivf_last_error(self.ctx) or b"").decode(errors="replace")
