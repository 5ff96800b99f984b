"""Small shared test utilities (no method arithmetic)."""
from __future__ import annotations

import numpy as np

from synth.corpus import Corpus, from_dense


def random_dense_corpus(N: int, D: int, density: float, seed: int, dup_rows: int = 0) -> tuple[np.ndarray, Corpus]:
    """Tiny dense non-negative matrix with unit-norm rows (fp32), then CSR.
    `dup_rows` rows are copies of earlier rows, to create exact score ties."""
    rng = np.random.default_rng(seed)
    X = np.zeros((N, D), dtype=np.float64)
    for i in range(N):
        m = rng.random(D) < density
        if not m.any():
            m[rng.integers(D)] = True
        X[i, m] = rng.random(m.sum()) + 0.05
    for t in range(dup_rows):
        X[N - 1 - t] = X[t]
    X /= np.linalg.norm(X, axis=1, keepdims=True)
    X32 = X.astype(np.float32)
    return X32, from_dense(X32)


def brute_force_scores(X32: np.ndarray, M: np.ndarray):
    """The plain definition, written independently of the oracle:
    rho_ij = sum over d = 0..D-1 (ascending) of x_i[d] * mu_j[d] in FP64, one
    Python float operation at a time. Zero products add exactly 0, so the sum
    equals the sparse sum taken in ascending term order bit for bit.
    Label = largest score, lowest index among equal scores."""
    N, D = X32.shape
    k = M.shape[0]
    rho = np.zeros((N, k), dtype=np.float64)
    for i in range(N):
        xi = [float(x) for x in X32[i]]
        for j in range(k):
            mj = M[j]
            acc = 0.0
            for d in range(D):
                acc = acc + xi[d] * float(mj[d])
            rho[i, j] = acc
    lab = np.empty(N, dtype=np.int32)
    for i in range(N):
        a = 0
        for j in range(1, k):
            if rho[i, j] > rho[i, a]:
                a = j
        lab[i] = a
    return lab, rho


def mean_direction(X32: np.ndarray, members: np.ndarray) -> np.ndarray:
    """mu = s / ||s|| with s the plain sum of the member rows (FP64)."""
    s = X32[members].astype(np.float64).sum(axis=0)
    return s / np.sqrt((s * s).sum())
