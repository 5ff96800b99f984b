"""ctypes front end of sivf_oracle.c (FP64 SIVF / IVF spherical k-means).

TEST INFRASTRUCTURE ONLY (see package docstring).

Paper map (Aoyama & Saito, arXiv 2103.16141):
  Oracle.assign()  -> Algorithm 2 (icp=False) / Algorithm 4 (icp=True) /
                      Algorithm 3 (icp="cbicp")
  Oracle.update()  -> Algorithm 5 (means, unit length, structured inverted file)
  Oracle.run()     -> Algorithm 1 loop until no label changes
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sivf_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "libsivf_oracle.so")
_lock = threading.Lock()
_lib = None


def build_library(force: bool = False) -> str:
    """Compile the oracle with gcc: -O2, OpenMP, no floating-point contraction
    (so x86 and Arm hosts round every multiply and add identically)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def bind(lib):
    """Declare the C signatures on a loaded oracle library."""
    i64, i32, p = ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p
    lib.orc_create.argtypes = [i64, i32, i32, p, p, p, p, ctypes.c_int]
    lib.orc_create.restype = p
    lib.orc_destroy.argtypes = [p]
    lib.orc_destroy.restype = None
    lib.orc_assign.argtypes = [p, p]
    lib.orc_assign.restype = ctypes.c_int
    lib.orc_update.argtypes = [p, p]
    lib.orc_update.restype = ctypes.c_int
    lib.orc_set_labels.argtypes = [p, p]
    lib.orc_set_labels.restype = ctypes.c_int
    lib.orc_iter.argtypes = [p]
    lib.orc_iter.restype = i32
    lib.orc_get_labels.argtypes = [p, p]
    lib.orc_get_scores.argtypes = [p, p, p, p]
    lib.orc_get_lambda.argtypes = [p, p]
    lib.orc_centroid_nnz.argtypes = [p]
    lib.orc_centroid_nnz.restype = i64
    lib.orc_get_centroids.argtypes = [p, p, p, p, p]
    lib.orc_if_nnz.argtypes = [p]
    lib.orc_if_nnz.restype = i64
    lib.orc_get_if.argtypes = [p, p, p, p, p]
    lib.orc_num_threads.restype = ctypes.c_int
    lib.orc_set_threads.argtypes = [ctypes.c_int]
    lib.orc_score_objects.argtypes = [p, p, i64, p, p, p]
    lib.orc_score_objects.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = bind(ctypes.CDLL(build_library()))
    return _lib


def _p(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


@dataclass
class AssignStats:
    changed: int
    n_moving: int        # clusters with lambda^[r] = 0 after this assignment
    simcalc: int         # similarity calculations (k per unfiltered object, #moving per filtered one)
    postings: int        # postings visited in the triple loop
    objective: float     # sum_i rho_{i, a(i)} against M^[r-1]
    filtered: int        # objects that took the filtered branch
    n_moving_prev: int   # #moving clusters at r-1 (the filtered objects' candidate count)
    r: int


@dataclass
class UpdateStats:
    objective: float     # sum_j ||s_j||, the objective after the update
    centroid_nnz: int
    empty: int


class Oracle:
    """One clustering instance held by the C oracle. Arrays passed in are kept
    referenced for the lifetime of the object (the C side borrows them)."""

    def __init__(self, corpus, k: int, init_ids: np.ndarray, icp=True, threads: int = 0, lib=None):
        """icp: False/0 unfiltered (Algorithm 2), True/1 SIVF (Algorithm 4),
        2 or "cbicp" IVF-CBICP (Algorithm 3), 3 or "relaxed" SIVF with the
        relaxed (own-similarity) filter."""
        self._lib = lib if lib is not None else _load()
        if threads:
            self._lib.orc_set_threads(int(threads))
        self.N, self.D, self.k = int(corpus.N), int(corpus.D), int(k)
        self._row_ptr = np.ascontiguousarray(corpus.row_ptr, dtype=np.int64)
        self._idx = np.ascontiguousarray(corpus.idx, dtype=np.int32)
        self._val = np.ascontiguousarray(corpus.val, dtype=np.float32)
        init = np.ascontiguousarray(init_ids, dtype=np.int32)
        if init.shape != (self.k,):
            raise ValueError("init_ids must have k entries")
        if icp == "cbicp" or (not isinstance(icp, bool) and icp == 2):
            mode = 2
        elif icp == "relaxed" or (not isinstance(icp, bool) and icp == 3):
            mode = 3
        else:
            mode = int(bool(icp))
        self._h = self._lib.orc_create(self.N, self.D, self.k, _p(self._row_ptr), _p(self._idx),
                                       _p(self._val), _p(init), mode)
        if not self._h:
            raise ValueError("oracle: invalid arguments or out of memory")
        self.icp = mode

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_destroy(h)
            self._h = None

    @staticmethod
    def threads() -> int:
        return int(_load().orc_num_threads())

    @property
    def iter(self) -> int:
        return int(self._lib.orc_iter(self._h))

    def assign(self) -> AssignStats:
        st = np.zeros(8, dtype=np.float64)
        if self._lib.orc_assign(self._h, _p(st)) != 0:
            raise MemoryError("oracle assign failed")
        return AssignStats(int(st[0]), int(st[1]), int(st[2]), int(st[3]), float(st[4]), int(st[5]),
                           int(st[6]), int(st[7]))

    def update(self) -> UpdateStats:
        st = np.zeros(3, dtype=np.float64)
        if self._lib.orc_update(self._h, _p(st)) != 0:
            raise MemoryError("oracle update failed")
        return UpdateStats(float(st[0]), int(st[1]), int(st[2]))

    def run(self, max_iter: int):
        """Algorithm 1 loop: assign + update until an assignment (r > 1)
        changes no label, or max_iter assignments. Returns per-iteration
        (AssignStats, UpdateStats or None on the converged step)."""
        hist = []
        for _ in range(max_iter):
            a = self.assign()
            if a.r > 1 and a.changed == 0:
                hist.append((a, None))
                break
            u = self.update()
            hist.append((a, u))
        return hist

    def set_labels(self, labels: np.ndarray) -> None:
        lab = np.ascontiguousarray(labels, dtype=np.int32)
        if lab.shape != (self.N,) or self._lib.orc_set_labels(self._h, _p(lab)) != 0:
            raise ValueError("labels out of range")

    def labels(self) -> np.ndarray:
        out = np.empty(self.N, dtype=np.int32)
        self._lib.orc_get_labels(self._h, _p(out))
        return out

    def scores(self):
        """(best, second, filtered) of the last assignment, FP64."""
        b = np.empty(self.N, dtype=np.float64)
        s = np.empty(self.N, dtype=np.float64)
        f = np.empty(self.N, dtype=np.uint8)
        self._lib.orc_get_scores(self._h, _p(b), _p(s), _p(f))
        return b, s, f

    def lam(self) -> np.ndarray:
        out = np.empty(self.k, dtype=np.uint8)
        self._lib.orc_get_lambda(self._h, _p(out))
        return out

    def centroids(self):
        """Cluster-major centroids: (off[k+1], term[nnz], val[nnz] fp64, ||s_j|| fp64[k])."""
        n = int(self._lib.orc_centroid_nnz(self._h))
        off = np.empty(self.k + 1, dtype=np.int64)
        term = np.empty(n, dtype=np.int32)
        val = np.empty(n, dtype=np.float64)
        sn = np.empty(self.k, dtype=np.float64)
        self._lib.orc_get_centroids(self._h, _p(off), _p(term), _p(val), _p(sn))
        return off, term, val, sn

    def inverted_file(self):
        """Structured inverted file: (off[D+1], mf0[D], cid[nnz], u[nnz] fp64)."""
        n = int(self._lib.orc_if_nnz(self._h))
        off = np.empty(self.D + 1, dtype=np.int64)
        mf0 = np.empty(self.D, dtype=np.int32)
        cid = np.empty(n, dtype=np.int32)
        u = np.empty(n, dtype=np.float64)
        self._lib.orc_get_if(self._h, _p(off), _p(mf0), _p(cid), _p(u))
        return off, mf0, cid, u

    def score_objects(self, ids: np.ndarray):
        """Unfiltered FP64 (label, best, second) for the given objects against
        the current centroids; no state change."""
        ids = np.ascontiguousarray(ids, dtype=np.int64)
        lab = np.empty(len(ids), dtype=np.int32)
        b = np.empty(len(ids), dtype=np.float64)
        s = np.empty(len(ids), dtype=np.float64)
        if self._lib.orc_score_objects(self._h, _p(ids), len(ids), _p(lab), _p(b), _p(s)) != 0:
            raise MemoryError("oracle scoring failed")
        return lab, b, s

    def dense_centroids(self) -> np.ndarray:
        """k x D dense FP64 copy of the current centroids (small cases only)."""
        off, term, val, _ = self.centroids()
        M = np.zeros((self.k, self.D), dtype=np.float64)
        for j in range(self.k):
            M[j, term[off[j]:off[j + 1]]] = val[off[j]:off[j + 1]]
        return M

