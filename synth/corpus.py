"""ctypes wrapper around corpus.c: seeded Zipf tf-idf corpora in CSR form."""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "corpus.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "libsynth.so")
_lock = threading.Lock()
_lib = None


def build_library(force: bool = False) -> str:
    """Compile corpus.c with gcc (OpenMP) into synth/_build/libsynth.so."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build_library())
            i64, i32, u64, dbl, p = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p
            lib.synth_lengths.argtypes = [i64, i32, dbl, dbl, i32, i32, u64, p]
            lib.synth_lengths.restype = None
            lib.synth_init_ids.argtypes = [i64, i32, u64, p]
            lib.synth_init_ids.restype = ctypes.c_int
            lib.synth_terms.argtypes = [i64, i32, dbl, u64, p, p, p]
            lib.synth_terms.restype = ctypes.c_int
            lib.synth_tfidf.argtypes = [i64, i32, p, p, p, p, p]
            lib.synth_tfidf.restype = i64
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


@dataclass
class Corpus:
    """CSR document-term matrix: int64 row_ptr[N+1], int32 idx[nnz], fp32 val[nnz]."""

    N: int
    D: int
    row_ptr: np.ndarray
    idx: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def row(self, i: int):
        b, e = int(self.row_ptr[i]), int(self.row_ptr[i + 1])
        return self.idx[b:e], self.val[b:e]


def generate(N: int, D: int, zipf_s: float, mu: float, sigma: float, lo: int, hi: int, seed: int) -> Corpus:
    """Seeded corpus: lognormal(mu, sigma) lengths clipped to [lo, hi], Zipf(zipf_s)
    terms without repeats, tf = 1 + Poisson(1), value = tf * ln(N/df), rows
    L2-normalised (fp64) and stored as fp32; zero-valued entries dropped."""
    lib = _load()
    lens = np.empty(N, dtype=np.int32)
    lib.synth_lengths(N, D, mu, sigma, lo, hi, seed, _ptr(lens))
    row_ptr = np.zeros(N + 1, dtype=np.int64)
    np.cumsum(lens, out=row_ptr[1:])
    nnz = int(row_ptr[-1])
    idx = np.empty(nnz, dtype=np.int32)
    tf = np.empty(nnz, dtype=np.int32)
    rc = lib.synth_terms(N, D, zipf_s, seed, _ptr(row_ptr), _ptr(idx), _ptr(tf))
    if rc != 0:
        raise MemoryError("synth_terms failed")
    val = np.empty(nnz, dtype=np.float32)
    new_ptr = np.empty(N + 1, dtype=np.int64)
    nnz2 = lib.synth_tfidf(N, D, _ptr(row_ptr), _ptr(idx), _ptr(tf), _ptr(val), _ptr(new_ptr))
    if nnz2 < 0:
        raise MemoryError("synth_tfidf failed")
    del tf
    if nnz2 != nnz:
        idx = idx[:nnz2].copy()
        val = val[:nnz2].copy()
    return Corpus(N=N, D=D, row_ptr=new_ptr, idx=idx, val=val)


def init_ids(N: int, k: int, seed: int) -> np.ndarray:
    """k distinct document ids drawn from [0, N) by a seeded partial Fisher-Yates."""
    lib = _load()
    out = np.empty(k, dtype=np.int32)
    rc = lib.synth_init_ids(N, k, seed, _ptr(out))
    if rc != 0:
        raise ValueError("k must be in [0, N]")
    return out


def from_dense(X: np.ndarray) -> Corpus:
    """CSR of a small dense non-negative matrix (test fixtures); zeros dropped."""
    X = np.asarray(X, dtype=np.float32)
    N, D = X.shape
    row_ptr = np.zeros(N + 1, dtype=np.int64)
    idx, val = [], []
    for i in range(N):
        nz = np.nonzero(X[i])[0]
        idx.extend(nz.tolist())
        val.extend(X[i, nz].tolist())
        row_ptr[i + 1] = len(idx)
    return Corpus(N=N, D=D, row_ptr=row_ptr, idx=np.asarray(idx, dtype=np.int32),
                  val=np.asarray(val, dtype=np.float32))
