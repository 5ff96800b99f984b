"""The error bound behind the near-tie re-score, checked against a model of
the scan's arithmetic on the CPU.

The assignment scan reads each term of an object either posting by posting
(sparse) or from a dense row of the term's values:
  - a sparse posting adds q = ceil(fl32(fl32(v * 2^31) * u~)) to an unsigned
    fixed-point score with quantum 2^-31;
  - the dense terms of each chunk of T staged terms are accumulated in FP32
    with a chain of fused multiply-adds, acc = fl32(vs * u~ + acc) in term
    order, and the chunk's sum then adds ceil(acc) once.
Here v is the object's value (vs = v * 2^31) and u~ the stored value: the
FP32 centroid value itself, its BF16 rounding, or its FP16 rounding of
u * 2^14 (clamped to the smallest subnormal, read back times 2^-14). Integer
sums are exact, so this model reproduces the scan's score bit for bit
whatever the order of the integer adds. The bound states, with n terms of
which nd are dense, and S = sum v,

    |rho~ - rho| <= E(rho~) = (c rho~ + a) / (1 - c),
    g = gamma_m = m 2^-24 / (1 - m 2^-24),  m = max(1, nd),
    c = eps + (1 + eps) g,  a = 2 n 2^-31 + (1 + g) eta S,

with eps = 0, 2^-8, 2^-11 and eta = 0, 0, 2^-38 for FP32, BF16, FP16, and rho
the exact score against the FP32 values. The test checks it on random rows,
on rows of many tiny values (where the FP16 subnormal term dominates), on
equal values and on single terms, with no, some and all terms dense and
several chunk sizes.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np
import pytest

Q = 2.0 ** -31
EPS = {"fp32": 0.0, "bf16": 2.0 ** -8, "fp16": 2.0 ** -11}
ETA = {"fp32": 0.0, "bf16": 0.0, "fp16": 2.0 ** -38}


def stored(u32: np.ndarray, prec: str) -> np.ndarray:
    """The FP32 value the scan multiplies by, for each FP32 centroid value."""
    if prec == "fp32":
        return u32
    if prec == "bf16":  # round to nearest even on the upper 16 bits
        b = u32.view(np.uint32).astype(np.uint64)
        r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
        return r.astype(np.uint32).view(np.float32)
    h = (u32 * np.float32(16384.0)).astype(np.float16)  # round to nearest even
    h = np.where((h == 0) & (u32 > 0), np.float16(2.0 ** -24), h)
    return h.astype(np.float32) * np.float32(2.0 ** -14)


def round_f32(x: Fraction) -> np.float32:
    """x rounded to the nearest FP32 value, ties to even (x >= 0, no overflow)."""
    f = np.float32(float(x))
    best = f
    for g in (np.nextafter(f, np.float32(0)), np.nextafter(f, np.float32(np.inf))):
        dg, db = abs(Fraction(float(g)) - x), abs(Fraction(float(best)) - x)
        if dg < db or (dg == db and (int(g.view(np.uint32)) & 1) == 0):
            best = g
    return np.float32(best)


def fma_f32(a: np.float32, b: np.float32, c: np.float32) -> np.float32:
    """fl32(a * b + c) with one rounding (a fused multiply-add)."""
    return round_f32(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c)))


def hybrid_score(v32: np.ndarray, u_st: np.ndarray, dense: np.ndarray, T: int) -> float:
    """The scan's fixed-point score: sparse terms one posting at a time, dense
    terms by an FP32 FMA chain per chunk of T staged terms."""
    vs = v32 * np.float32(2.0 ** 31)  # exact: power-of-two scaling
    total = 0
    for c0 in range(0, len(v32), T):
        acc, used = np.float32(0.0), False
        for h in range(c0, min(c0 + T, len(v32))):
            if dense[h]:
                acc = fma_f32(vs[h], u_st[h], acc)
                used = True
            else:
                total += int(np.ceil(np.float64(vs[h] * u_st[h])))  # one FP32 rounding, then ceil
        if used:
            total += int(np.ceil(np.float64(acc)))
    assert total < 2 ** 32, "the unsigned 32-bit score would overflow"
    return total * Q


def bound(x: float, n: int, nd: int, S: float, prec: str) -> float:
    eps, eta = EPS[prec], ETA[prec]
    m = max(1, nd)
    g = m * 2.0 ** -24 / (1 - m * 2.0 ** -24)
    c = eps + (1 + eps) * g
    a = 2 * n * Q + (1 + g) * eta * S
    return (c * x + a) / (1 - c)


def unit(x: np.ndarray) -> np.ndarray:
    return (x / np.sqrt((x.astype(np.float64) ** 2).sum())).astype(np.float32)


def cases(rng):
    for n in (1, 2, 7, 60, 190, 1000):
        for _ in range(12):
            v = unit(rng.pareto(1.5, n) + 1e-3)
            u = unit(rng.pareto(1.2, n) + 1e-4) * np.float32(rng.uniform(0.05, 1.0))
            yield v, u
    for n in (50, 400):  # tiny centroid values: FP16 subnormals and the clamp
        for scale in (1e-6, 1e-9, 1e-12):
            v = unit(rng.random(n) + 0.1)
            u = (rng.random(n).astype(np.float32) * np.float32(scale)).astype(np.float32)
            yield v, u
    for n in (16, 256):  # equal values
        yield unit(np.ones(n)), unit(np.ones(n))
    yield np.array([1.0], np.float32), np.array([1.0], np.float32)


def masks(rng, n):
    yield "none", np.zeros(n, bool)
    yield "all", np.ones(n, bool)
    yield "half", rng.random(n) < 0.5


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16"])
def test_hybrid_score_within_the_derived_bound(prec):
    rng = np.random.default_rng({"fp32": 1, "bf16": 2, "fp16": 3}[prec])
    worst = {"none": 0.0, "all": 0.0, "half": 0.0}
    for v, u in cases(rng):
        rho = float((v.astype(np.float64) * u.astype(np.float64)).sum())
        S = float(v.astype(np.float64).sum())
        for name, dense in masks(rng, len(v)):
            for T in (32, 64, 512):
                x = hybrid_score(v, stored(u, prec), dense, T)
                E = bound(x, len(v), int(dense.sum()), S, prec)
                assert abs(x - rho) <= E, (prec, name, T, len(v), x, rho, E)
                if E > 0:
                    worst[name] = max(worst[name], abs(x - rho) / E)
    # the bound is exercised, not vacuous, for the sparse form; the dense
    # chain's gamma term is a worst case that random rows reach only in part
    assert worst["none"] > 0.01, worst
    assert worst["all"] > 1e-3 and worst["half"] > 1e-3, worst


def test_bound_catches_a_too_small_epsilon():
    """The model is sensitive: with BF16 postings but the FP32 constants the
    bound fails on some row (so the test above would catch a wrong eps)."""
    rng = np.random.default_rng(4)
    failed = False
    for v, u in cases(rng):
        rho = float((v.astype(np.float64) * u.astype(np.float64)).sum())
        S = float(v.astype(np.float64).sum())
        x = hybrid_score(v, stored(u, "bf16"), np.zeros(len(v), bool), 64)
        if abs(x - rho) > bound(x, len(v), 0, S, "fp32"):
            failed = True
            break
    assert failed


def test_dense_chain_needs_its_gamma_term():
    """With every term dense in one chunk (one ceil), FP32 rows, and only the
    single-rounding relative term 2^-24 plus that one quantum, the error
    exceeds the allowance on some row of many terms: the chain's gamma_nd
    term is needed (the bound's 2 n 2^-31 slack would otherwise hide it)."""
    rng = np.random.default_rng(6)
    failed = False
    for _ in range(10):
        n = 3000
        v = unit(rng.random(n) + 0.5)
        u = unit(rng.random(n) + 0.5)
        rho = float((v.astype(np.float64) * u.astype(np.float64)).sum())
        x = hybrid_score(v, u, np.ones(n, bool), 3000)
        assert abs(x - rho) <= bound(x, n, n, float(v.astype(np.float64).sum()), "fp32")
        if abs(x - rho) > 2.0 ** -24 * x + Q:
            failed = True
            break
    assert failed


def test_fma_model_is_one_rounding():
    """fma_f32 rounds once: it differs from the two-rounding form on a case
    built for it, and agrees with exact float64 arithmetic where that is
    exact."""
    a = np.float32(1.0 + 2.0 ** -12)
    b = np.float32(1.0 + 2.0 ** -12)
    c = np.float32(-1.0)
    # a*b = 1 + 2^-11 + 2^-24: exact fma keeps the 2^-24 bit, a rounded product loses it
    assert float(fma_f32(a, b, c)) == 2.0 ** -11 + 2.0 ** -24
    assert float(np.float32(a * b) + c) == 2.0 ** -11
    x, y, z = np.float32(3.0), np.float32(0.5), np.float32(0.25)
    assert float(fma_f32(x, y, z)) == 1.75


def test_bf16_model_rounds_like_torch():
    """The BF16 rounding of the model (nearest, ties to even) is torch's."""
    import torch
    rng = np.random.default_rng(5)
    u = (rng.random(100_000) * 10.0 ** rng.integers(-12, 1, 100_000)).astype(np.float32)
    ref = torch.from_numpy(u).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(stored(u, "bf16"), ref)
