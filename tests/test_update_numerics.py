"""The arithmetic of the update step's row passes, checked against a model on
the CPU.

The dense-form update keeps, per cluster j and term, the integer sum
S = sum of ceil(x * 2^s) over the members; the row's norm ||S|| stays below
2^63 (at most N members of unit norm, s = 62 - bits(N)). Pass 1 forms
||S||^2 exactly as a 128-bit integer: each thread adds the squares of its
entries into (hi, lo) 64-bit halves with a carry, and the block adds the
threads' pairs in a fixed tree, again with carries; ||s_j|| is then
sqrt((double(hi) 2^64 + double(lo)) 2^-2s) in FP64. Pass 2 writes each
centroid value u = S 2^-s / ||s_j|| in FP32 as

    f  = fl32(2^-s / ||s_j||)                       (FP64 division, one FP32 rounding)
    fs = fl32(fl32(S >> 32) * 2^32 + fl32(S mod 2^32))  (one fused multiply-add)
    u~ = fl32(fs * f),

at most four roundings of 2^-24 each, so |u~ / u - 1| < 2.4e-7. The tests
run that model in exact integer arithmetic and check: the 128-bit sum equals
the exact sum (with low halves that wrap on about half of the adds, and a
model without the carries fails), the norm is within a few FP64 roundings, and every value is within
2.4e-7 of the exact one, with an observed error large enough that the bound
is not slack.
"""
from __future__ import annotations

from decimal import Decimal, getcontext

import numpy as np
import pytest

M64 = (1 << 64) - 1
THREADS = 256  # block size of the row passes


def u128_block_sum_of_squares(vals: list[int]) -> tuple[int, int]:
    """(hi, lo) of sum v^2 as the kernel forms it: strided per-thread sums
    with a carry, then a fixed-tree reduction of the pairs with carries."""
    hi = [0] * THREADS
    lo = [0] * THREADS
    for t in range(THREADS):
        for p in range(t, len(vals), THREADS):
            u = vals[p]
            sq_lo = (u * u) & M64
            sq_hi = (u * u) >> 64  # __umul64hi
            lo[t] = (lo[t] + sq_lo) & M64
            hi[t] += sq_hi + (1 if lo[t] < sq_lo else 0)
    s = THREADS // 2
    while s > 0:
        for t in range(s):
            l = (lo[t] + lo[t + s]) & M64
            hi[t] += hi[t + s] + (1 if l < lo[t] else 0)
            lo[t] = l
        s //= 2
    return hi[0], lo[0]


def rn32_int(x: int) -> float:
    """x > 0 rounded to the nearest FP32 value, ties to even (exactly)."""
    if x == 0:
        return 0.0
    b = x.bit_length()
    if b <= 24:
        return float(x)
    shift = b - 24
    q, r = divmod(x, 1 << shift)
    half = 1 << (shift - 1)
    if r > half or (r == half and q & 1):
        q += 1
    return float(q << shift)


def fp32_value(S: int, f: np.float32) -> float:
    hi, lo = S >> 32, S & 0xFFFFFFFF
    fh = rn32_int(hi)  # __uint2float_rn
    fl = rn32_int(lo)
    fs = rn32_int(int(fh) * (1 << 32) + int(fl))  # fmaf: exact product and sum, one rounding
    return float(np.float32(np.float64(fs) * np.float64(f)))  # the product is exact in FP64


def row(rng, n: int, bits: int) -> list[int]:
    return [int(x) for x in rng.integers(1, 1 << bits, size=n, dtype=np.uint64)]


@pytest.mark.parametrize("bits", [20, 40, 52, 57])
def test_u128_sum_of_squares_is_exact(bits):
    # ||S|| < 2^63 (S sums at most N values of at most 2^s each, s = 62 - bits(N)):
    # 3000 entries of up to 57 bits keep the sum of squares below 2^126
    rng = np.random.default_rng(bits)
    vals = row(rng, 3000, bits)
    hi, lo = u128_block_sum_of_squares(vals)
    assert (hi << 64) + lo == sum(v * v for v in vals)
    assert hi < 1 << 62


def test_u128_sum_carries():
    # 1024 entries just below 2^58: the sum of squares is just below 2^126 and
    # the 64-bit low halves wrap on about half of the adds
    vals = [(1 << 58) - 1 - 977 * k for k in range(1024)]
    hi, lo = u128_block_sum_of_squares(vals)
    assert (hi << 64) + lo == sum(v * v for v in vals)
    assert (1 << 61) <= hi < 1 << 62


def test_dropping_the_carry_is_caught():
    vals = [(1 << 58) - 1 - 977 * k for k in range(512)]
    exact = sum(v * v for v in vals)
    # the same tree without the carries of the low halves
    hi = [0] * THREADS
    lo = [0] * THREADS
    for t in range(THREADS):
        for p in range(t, len(vals), THREADS):
            u = vals[p]
            lo[t] = (lo[t] + ((u * u) & M64)) & M64
            hi[t] += (u * u) >> 64
    s = THREADS // 2
    while s > 0:
        for t in range(s):
            lo[t] = (lo[t] + lo[t + s]) & M64
            hi[t] += hi[t + s]
        s //= 2
    assert (hi[0] << 64) + lo[0] != exact


@pytest.mark.parametrize("bits,shift", [(30, 20), (48, 40), (57, 43)])
def test_fp32_values_within_the_stated_bound(bits, shift):
    getcontext().prec = 60
    rng = np.random.default_rng(1000 + bits)
    vals = row(rng, 2000, bits)
    hi, lo = u128_block_sum_of_squares(vals)
    inv_scale = 2.0 ** -shift
    nrm = np.sqrt((float(hi) * 18446744073709551616.0 + float(lo)) * (inv_scale * inv_scale))
    exact_norm = Decimal(sum(v * v for v in vals)).sqrt()  # ||S||, unscaled
    assert abs(Decimal(nrm) / (exact_norm * Decimal(inv_scale)) - 1) < Decimal(1e-15)
    f = np.float32(inv_scale / nrm)
    worst = Decimal(0)
    for S in vals:
        got = Decimal(fp32_value(S, f))
        want = Decimal(S) / exact_norm
        worst = max(worst, abs(got / want - 1))
    assert worst < Decimal(2.4e-7)
    assert worst > Decimal(2.0 ** -25)  # several roundings do show: the bound is not slack by orders


def test_fp32_values_whose_halves_both_round():
    # both 32-bit halves need more than 24 bits, so each conversion rounds
    f = np.float32(2.0 ** -63 * 1.2345)
    for S in [(1 << 63) - 1, (1 << 62) + (1 << 31) + 12345, ((1 << 32) - 1) << 31 | ((1 << 31) - 1)]:
        want = Decimal(S) * Decimal(float(f))
        got = Decimal(fp32_value(S, f))
        assert abs(got / want - 1) < Decimal(2.4e-7)
