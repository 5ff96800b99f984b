"""Workload recipes: the five synthetic corpora that stand in for the paper's
PubMed (D ~ 140K, ~59 nnz/doc) and NYT (~226 nnz/doc) sets (Section 5.1).

Each entry gives the generator parameters, k, the iteration cap and the
posting precision the workload is run with.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, replace


@dataclass(frozen=True)
class Workload:
    name: str
    N: int
    D: int
    zipf_s: float
    mu: float
    sigma: float
    lo: int
    hi: int
    k: int
    max_iter: int
    precision: str  # "fp32" | "bf16" | "fp16"
    seed: int

    @property
    def init_seed(self) -> int:
        return self.seed * 1000003 + 17

    def scaled(self, **kw) -> "Workload":
        return replace(self, **kw)


def _mu_for_mean(mean: float, sigma: float) -> float:
    return math.log(mean) - sigma * sigma / 2.0


CONFIGS = {
    # C1: plain SIVF, FP32 vs the FP64 oracle, run to convergence (cap 30)
    "c1": Workload("c1", 2_000, 5_000, 1.1, 3.5, 0.6, 5, 300, 50, 30, "fp32", 1),
    # C2: plain FP32 SIVF at medium scale (NYT-like density)
    "c2": Workload("c2", 300_000, 100_000, 1.05, 5.0, 0.7, 10, 3000, 1_000, 50, "fp32", 2),
    # C3: mixed precision, BF16 postings + FP32 re-score
    "c3": Workload("c3", 1_000_000, 140_000, 1.1, 4.2, 0.8, 5, 3000, 10_000, 50, "bf16", 3),
    # C5: large single instance, BF16 postings
    "c5": Workload("c5", 8_000_000, 140_000, 1.1, _mu_for_mean(60.0, 0.8), 0.8, 5, 3000, 20_000, 20, "bf16", 5),
    # the C5 regime scaled to 1/16 of its objects (k = 20,000 kept; 30M nnz,
    # a 0.25 GB CSR, still larger than L2): the case kernel profiles capture
    "c5s": Workload("c5s", 500_000, 140_000, 1.1, _mu_for_mean(60.0, 0.8), 0.8, 5, 3000, 20_000, 20, "bf16", 55),
}


def small_config(name: str = "c1") -> Workload:
    return CONFIGS[name]


class _SplitMix64:
    """SplitMix64 (Steele, Lea & Flood 2014), for seeded instance parameters."""

    def __init__(self, seed: int):
        self.s = seed & 0xFFFFFFFFFFFFFFFF

    def next(self) -> int:
        self.s = (self.s + 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF
        z = self.s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & 0xFFFFFFFFFFFFFFFF
        return z ^ (z >> 31)

    def unif(self) -> float:
        return ((self.next() >> 11) + 0.5) / float(1 << 53)

    def log_uniform(self, a: float, b: float) -> float:
        return math.exp(math.log(a) + (math.log(b) - math.log(a)) * self.unif())


def batched_instances(n_inst: int = 64, scale: float = 1.0, max_iter: int = 50) -> list[Workload]:
    """C4: independent corpora with seeds 0..n_inst-1. N log-uniform in
    [5K, 200K], D log-uniform in [20K, 100K], mean nnz/doc uniform in
    [30, 250] (sigma 0.7), k log-uniform in [16, 2000]; FP16 postings.
    `scale` shrinks N (and caps k at N) for small test cases."""
    out = []
    for s in range(n_inst):
        g = _SplitMix64(0xC4C4 + s)
        N = int(round(g.log_uniform(5_000, 200_000) * scale))
        D = int(round(g.log_uniform(20_000, 100_000)))
        mean = 30.0 + 220.0 * g.unif()
        k = int(round(g.log_uniform(16, 2_000)))
        N = max(N, 8)
        k = max(1, min(k, N))
        out.append(Workload(f"c4_{s}", N, D, 1.1, _mu_for_mean(mean, 0.7), 0.7, 5, 3000, k, max_iter, "fp16", s))
    return out
