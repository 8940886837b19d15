"""Seeded synthetic workloads: integrand families, parameter draws, configs.

This module holds no arithmetic of the integration method.  It only draws
integrand parameters from a counter-free splitmix64 stream (published by
Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014; constants as in Vigna's reference implementation) and names the
workloads.  Both the CUDA path and the CPU oracle receive the same drawn
parameter vectors through their own front ends.

The paper evaluates on Genz-family integrands with fixed parameters
(Sec. 4.1, Sec. 4.2).  The synthetic instances below stand in for that suite:
same families, parameters drawn from the stated uniform ranges.

Parameter layouts (all float64, dimension n):
  PRODUCT_PEAK  prod 1/(c_j^-2 + (x_j - w_j)^2)    [c_0..c_{n-1}, w_0..w_{n-1}]
  GAUSSIAN      exp(-sum a_j^2 (x_j - w_j)^2)      [a_0..a_{n-1}, w_0..w_{n-1}]
  OSCILLATORY   cos(2 pi u + sum a_j x_j)          [u, a_0..a_{n-1}]
  CORNER_PEAK   (1 + sum a_j x_j)^-(n+1)           [a_0..a_{n-1}]
  C0            exp(-sum a_j |x_j - w_j|)          [a_0..a_{n-1}, w_0..w_{n-1}]
  DISCONTINUOUS exp(sum a_j x_j) if all x_j < w_j    [a_0..a_{n-1}, w_0..w_{n-1}]
  BOX_POWER     (sum x_j^2)^q                      [q]
"""
from __future__ import annotations

from dataclasses import dataclass, field

PRODUCT_PEAK, GAUSSIAN, OSCILLATORY, CORNER_PEAK, C0, DISCONTINUOUS, BOX_POWER = 0, 1, 2, 3, 4, 5, 6
FAMILY_NAMES = {PRODUCT_PEAK: "product_peak", GAUSSIAN: "gaussian", OSCILLATORY: "oscillatory",
                CORNER_PEAK: "corner_peak", C0: "c0", DISCONTINUOUS: "discontinuous", BOX_POWER: "box_power"}
BASE_SEED = 2104
_MASK = (1 << 64) - 1


class SplitMix64:
    """splitmix64 stream; uniform() returns the top 53 bits scaled to [0, 1)."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        u = (self.next_u64() >> 11) * (1.0 / (1 << 53))
        return lo + (hi - lo) * u


def param_count(family: int, n: int) -> int:
    return {PRODUCT_PEAK: 2 * n, GAUSSIAN: 2 * n, OSCILLATORY: n + 1, CORNER_PEAK: n, C0: 2 * n,
            DISCONTINUOUS: 2 * n, BOX_POWER: 1}[family]


# default parameter ranges per family: list of (count_fn, lo, hi) in draw order
_RANGES = {
    PRODUCT_PEAK: [("n", 5.0, 10.0), ("n", 0.2, 0.8)],
    GAUSSIAN: [("n", 5.0, 15.0), ("n", 0.0, 1.0)],
    OSCILLATORY: [("1", 0.0, 1.0), ("n", 1.0, 5.0)],
    CORNER_PEAK: [("n", 0.5, 2.0)],
    C0: [("n", 1.0, 5.0), ("n", 0.0, 1.0)],
    DISCONTINUOUS: [("n", 1.0, 5.0), ("n", 0.2, 0.9)],
    BOX_POWER: [("1", 1.0, 11.0)],
}


def draw_params(family: int, n: int, seed: int, ranges=None) -> list[float]:
    """Draw a parameter vector: each block (first all i of the first vector,
    then the second) from U[lo, hi)."""
    rng = SplitMix64(seed)
    out: list[float] = []
    for cnt, lo, hi in (ranges or _RANGES[family]):
        k = n if cnt == "n" else int(cnt)
        out.extend(rng.uniform(lo, hi) for _ in range(k))
    return out


@dataclass
class Workload:
    name: str
    family: int
    dim: int
    epsrel: float
    params: list[float]
    max_regions: int
    relerr_filter: int = 1
    epsabs: float = 1e-20
    notes: str = ""
    extra: dict = field(default_factory=dict)


def config_workloads() -> dict[str, Workload]:
    """The five single-integral workloads (seeded, synthetic)."""
    return {
        "product_peak_d3": Workload("product_peak_d3", PRODUCT_PEAK, 3, 1e-3,
                                    draw_params(PRODUCT_PEAK, 3, BASE_SEED + 1), 100_000),
        "gaussian_d5": Workload("gaussian_d5", GAUSSIAN, 5, 1e-7,
                                draw_params(GAUSSIAN, 5, BASE_SEED + 2), 40_000_000),
        "oscillatory_d6": Workload("oscillatory_d6", OSCILLATORY, 6, 1e-8,
                                   draw_params(OSCILLATORY, 6, BASE_SEED + 3), 40_000_000, relerr_filter=0,
                                   notes="sign-changing integrand: rel-err filtering off (Sec. 3.5.1)"),
        # the same integral at 1e-10: at 1e-8 it converges with at most 6.6e4
        # active regions, at 1e-10 its active set reaches 4.2e6, the
        # 1e6..1e7 range the 6-D oscillatory workload is specified for
        "oscillatory_d6_1e-10": Workload("oscillatory_d6_1e-10", OSCILLATORY, 6, 1e-10,
                                         draw_params(OSCILLATORY, 6, BASE_SEED + 3), 40_000_000, relerr_filter=0,
                                         notes="oscillatory_d6 at a tolerance whose active set reaches 1e6..1e7"),
        "corner_peak_d8": Workload("corner_peak_d8", CORNER_PEAK, 8, 1e-6,
                                   draw_params(CORNER_PEAK, 8, BASE_SEED + 4), 400_000_000),
        "c0_d8": Workload("c0_d8", C0, 8, 1e-6, draw_params(C0, 8, BASE_SEED + 5), 400_000_000),
        "gaussian_d6_grad": Workload("gaussian_d6_grad", GAUSSIAN, 6, 1e-7,
                                     draw_params(GAUSSIAN, 6, BASE_SEED + 6, [("n", 5.0, 15.0), ("n", 0.2, 0.8)]),
                                     40_000_000, notes="differentiation: theta = (a_1..a_6, w_1..w_6)"),
    }


def random_dyadic_regions(n: int, m: int, seed: int, max_level: int = 12):
    """m random dyadic boxes in [0,1]^n (lower = k 2^-l, width = 2^-l per
    axis), as two m x n lists.  Used to feed identical region sets to both
    evaluate implementations."""
    rng = SplitMix64(seed)
    lower, width = [], []
    for _ in range(m):
        lo, wd = [], []
        for _ in range(n):
            lvl = int(rng.uniform(0, max_level + 1))
            k = int(rng.uniform(0, 1 << lvl))
            lo.append(k / (1 << lvl))
            wd.append(1.0 / (1 << lvl))
        lower.append(lo)
        width.append(wd)
    return lower, width


def batch_workloads(count: int = 4096, seed: int = BASE_SEED + 100) -> list[Workload]:
    """Independent integrals for the batched form: dimension uniform in
    {3..8}, family uniform over the five families, epsrel uniform in
    {1e-4, 1e-6, 1e-8}, parameters from each family's ranges with a per-item
    seed (seed + 1 + index).  Rel-err filtering is off for the oscillatory
    family (sign-changing)."""
    rng = SplitMix64(seed)
    out = []
    for i in range(count):
        dim = 3 + int(rng.uniform(0, 6))
        fam = int(rng.uniform(0, 5))
        tau = (1e-4, 1e-6, 1e-8)[int(rng.uniform(0, 3))]
        out.append(Workload(f"batch_{i}", fam, dim, tau, draw_params(fam, dim, seed + 1 + i), 0,
                            relerr_filter=0 if fam == OSCILLATORY else 1))
    return out


def paper_integrands() -> dict[str, Workload]:
    """The paper's fixed-parameter test integrands (Sec. 4.1) on their
    dimensions, mapped onto the families; epsrel and pool set per use."""
    def w(name, fam, n, params, relerr=1):
        return Workload(name, fam, n, 1e-3, params, 10_000_000, relerr_filter=relerr)
    out = {
        "f1_d8": w("f1_d8", OSCILLATORY, 8, [0.0] + [float(i) for i in range(1, 9)], relerr=0),
        "f2_d6": w("f2_d6", PRODUCT_PEAK, 6, [50.0] * 6 + [0.5] * 6),
        "f3_d3": w("f3_d3", CORNER_PEAK, 3, [1.0, 2.0, 3.0]),
        "f3_d8": w("f3_d8", CORNER_PEAK, 8, [float(i) for i in range(1, 9)]),
        "f4_d5": w("f4_d5", GAUSSIAN, 5, [25.0] * 5 + [0.5] * 5),
        "f4_d8": w("f4_d8", GAUSSIAN, 8, [25.0] * 8 + [0.5] * 8),
        "f5_d5": w("f5_d5", C0, 5, [10.0] * 5 + [0.5] * 5),
        "f5_d8": w("f5_d8", C0, 8, [10.0] * 8 + [0.5] * 8),
        "f6_d6": w("f6_d6", DISCONTINUOUS, 6, [float(i + 4) for i in range(1, 7)] +
                   [(3 + i) / 10 for i in range(1, 7)]),
        "f7_d8": w("f7_d8", BOX_POWER, 8, [11.0]),
        "f8_d8": w("f8_d8", BOX_POWER, 8, [7.5]),
    }
    return out
