"""The error bound behind the near-tie re-score, checked against a model of
the scan's arithmetic on the CPU.

Each posting of the assignment scan adds q = ceil(fl32(fl32(v * 2^31) * u~))
to an unsigned fixed-point score with quantum 2^-31, where v is the object's
value and u~ the stored posting value: the FP32 centroid value itself, its
BF16 rounding, or its FP16 rounding of u * 2^14 (clamped to the smallest
subnormal, read back times 2^-14). Integer sums are exact, so this model
reproduces the scan's score bit for bit whatever the summation order. The
bound states, with n terms and S = sum v,

    |rho~ - rho| <= E(rho~) = (c rho~ + a) / (1 - c),
    c = 2^-24 (1 + eps) + eps,  a = n 2^-31 + (1 + 2^-24) eta S,

with eps = 0, 2^-8, 2^-11 and eta = 0, 0, 2^-38 for FP32, BF16, FP16, and
rho the exact score against the FP32 values. The test checks it on random
rows, on rows of many tiny values (where the FP16 subnormal term dominates),
on equal values and on single terms.
"""
from __future__ import annotations

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


def fixed_point_score(v32: np.ndarray, u_st: np.ndarray) -> float:
    vs = v32 * np.float32(2.0 ** 31)          # exact: power-of-two scaling
    prod = vs * u_st                          # one FP32 rounding
    q = np.ceil(prod.astype(np.float64)).astype(np.uint64)
    total = int(q.sum())
    assert total < 2 ** 32, "the unsigned 32-bit score would overflow"
    return total * Q


def bound(x: float, n: int, S: float, prec: str) -> float:
    eps, eta = EPS[prec], ETA[prec]
    c = 2.0 ** -24 * (1 + eps) + eps
    a = n * Q + (1 + 2.0 ** -24) * eta * S
    return (c * x + a) / (1 - c)


def unit(x: np.ndarray) -> np.ndarray:
    return (x / np.sqrt((x.astype(np.float64) ** 2).sum())).astype(np.float32)


def cases(rng):
    for n in (1, 2, 7, 60, 190, 1000, 3000):
        for _ in range(40):
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


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16"])
def test_fixed_point_score_within_the_derived_bound(prec):
    rng = np.random.default_rng({"fp32": 1, "bf16": 2, "fp16": 3}[prec])
    worst = 0.0
    for v, u in cases(rng):
        rho = float((v.astype(np.float64) * u.astype(np.float64)).sum())
        x = fixed_point_score(v, stored(u, prec))
        E = bound(x, len(v), float(v.astype(np.float64).sum()), prec)
        assert abs(x - rho) <= E, (prec, len(v), x, rho, E)
        if E > 0:
            worst = max(worst, abs(x - rho) / E)
    assert worst > 0.01  # the bound is exercised, not vacuous


def test_bound_catches_a_too_small_epsilon():
    """The model is sensitive: with BF16 postings but the FP32 constants the
    bound fails on some row (so the test above would catch a wrong eps)."""
    rng = np.random.default_rng(4)
    failed = False
    for v, u in cases(rng):
        rho = float((v.astype(np.float64) * u.astype(np.float64)).sum())
        x = fixed_point_score(v, stored(u, "bf16"))
        if abs(x - rho) > bound(x, len(v), float(v.sum()), "fp32"):
            failed = True
            break
    assert failed


def test_bf16_model_rounds_like_torch():
    """The BF16 rounding of the model (nearest, ties to even) is torch's."""
    import torch
    rng = np.random.default_rng(5)
    u = (rng.random(100_000) * 10.0 ** rng.integers(-12, 1, 100_000)).astype(np.float32)
    ref = torch.from_numpy(u).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(stored(u, "bf16"), ref)
