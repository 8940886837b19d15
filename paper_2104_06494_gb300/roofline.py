"""Algorithmic work of the Evaluate kernel, for its roofline.

Evaluate is bound by the FP64 pipe (GB300 issues about 2 FP64 FMA per clock
per SM), so its roofline is FP64 throughput.  The counts below follow the
kernel's loop structure (csrc/pagani_eval.cuh) operation by operation, per
sibling pair (one thread):

* the per-axis factor table: 11 coordinate codes on n + 1 axes (the pair
  shares n - 1 axes, and the split axis is patched for the right region).
  With the per-axis factor cache (levels <= 11) these entries are loads, not
  FP64 work; the cache fill (one level per iteration, n 2^L 11 factors) is a
  separate kernel, counted by `cache_fill_work`;
* per region: prefix/suffix partial products, the one-axis, pair, triple and
  vertex orbits (one product or sum per point from shared partials), the
  nine generator sums, the fourth differences and their noise floors, rule
  and null-rule weighting,
  the noise floors, the error formula and the split axis;
* per pair: the two-level refinement; per region: the compensated partial
  sums and Rel-Err-Classify.

flops count an FMA as 2 and every other add/mul as 1; `inst` counts FP64
arithmetic instructions (an FMA is one).  Library calls (exp, sincos,
division, sqrt, pow: CUDA's own implementations) are counted separately and
never converted into flops.
"""
from __future__ import annotations

from collections import Counter

PRODUCT_PEAK, GAUSSIAN, OSCILLATORY, CORNER_PEAK, C0, DISCONTINUOUS, BOX_POWER = 0, 1, 2, 3, 4, 5, 6


def num_points(n: int) -> int:
    return 1 + 8 * n + 6 * n * (n - 1) + 4 * n * (n - 1) * (n - 2) // 3 + 2 ** n


def _pow_mults(e: int) -> int:
    """Multiplications of the binary powering r^e as the kernel writes it
    (the first multiply into y = 1 folds away)."""
    mults, first = 0, True
    while e > 0:
        if e & 1:
            mults += 0 if first else 1
            first = False
        if e > 1:
            mults += 1
        e >>= 1
    return mults


def _box_power_outer(q: float) -> Counter:
    """(s)^q as the box-power kernel forms it: binary powering for integer
    and half-integer q (one multiply per bit and per set bit, plus a square
    root and a multiply for the half), a library pow otherwise."""
    c = Counter()
    if 2 * q == int(2 * q) and q < 64:
        k = int(q)
        c["flops"] += k.bit_length() + bin(k).count("1")
        c["inst"] += k.bit_length() + bin(k).count("1")
        if 2 * q != 2 * k:
            c["sqrt"] += 1
            c["flops"] += 1
            c["inst"] += 1
    else:
        c["pow"] += 1
    return c


def region_points_work(family: int, n: int, q: float = 11.0) -> Counter:
    """FP64 work of the rule sums of one region (rule_sums in the kernel);
    q is the box-power exponent."""
    c = Counter()
    cplx = family == OSCILLATORY
    corner = family == CORNER_PEAK
    box = family == BOX_POWER
    additive = corner or box
    base_identity = family in (PRODUCT_PEAK, GAUSSIAN, C0, DISCONTINUOUS)

    def mul(k=1):
        if cplx:          # (a.x b.x - a.y b.y, a.x b.y + a.y b.x): 2 MUL + 2 FMA
            c["flops"] += 6 * k
            c["inst"] += 4 * k
        else:             # one MUL (or ADD for the corner peak's sums)
            c["flops"] += k
            c["inst"] += k

    def outer(k=1):       # corner peak: 1 / s, then r^(n+1); box power: s^q
        if box:
            for key, v in _box_power_outer(q).items():
                c[key] += v * k
            return
        c["div"] += k
        pm = _pow_mults(n + 1)
        c["flops"] += pm * k
        c["inst"] += pm * k

    def last(k=1):
        c["points"] += k  # a rule point's value formed
        if cplx:          # real part only: 1 MUL + 1 FMA
            c["flops"] += 3 * k
            c["inst"] += 2 * k
        else:
            c["flops"] += k
            c["inst"] += k
        if additive:
            outer(k)

    def add(k=1):
        c["flops"] += k
        c["inst"] += k

    def acc(k=1):         # S += f(point) formed from its last two factors
        c["points"] += k
        if cplx:          # 2 FMA
            c["flops"] += 4 * k
            c["inst"] += 2 * k
        elif additive:    # S + outer(a + b)
            add(2 * k)
            outer(k)
        else:             # 1 FMA
            c["flops"] += 2 * k
            c["inst"] += k

    # prefix and suffix partial products
    mul(n - 1 if base_identity else n)
    mul(max(n - 2, 0))
    if additive:
        outer(1)          # f at the centre
    # one-axis orbits and fourth differences
    for j in range(n):
        if j < n - 1:
            mul()
        acc(4)            # the l1 and l3 points
        if cplx or additive:
            last(4)       # the l2 and lp points (also used by D_j)
            add(4)        # their pair sums and the two generator sums
        else:
            last(2)       # one point of each pair, the other fused into
            acc(2)        # the pair sum (D_j needs only the sums)
            add(2)        # the two generator sums
        c["flops"] += 6   # (sp - 2 f0) - q (s2 - 2 f0): 3 FMA
        c["inst"] += 3
        if cplx:          # its noise floor over |values|: 3 ADD, 2 FMA (|x| is free)
            c["flops"] += 7
            c["inst"] += 5
        else:             # positive values: 3 FMA
            c["flops"] += 6
            c["inst"] += 3
    # axis pairs
    for j in range(n - 1):
        for k in range(j + 1, n):
            if k > j + 1:
                mul()
            if k < n - 1:
                mul()
            mul(4)
            acc(12)
    # axis triples
    for j in range(n - 2):
        for k in range(j + 1, n - 1):
            if k > j + 1:
                mul()
            mul(2 + 4)
            mid_id = True
            for l in range(k + 1, n):
                if l > k + 1:
                    if not mid_id:
                        mul()
                    mid_id = False
                if l == n - 1:
                    c_id = mid_id
                else:
                    if not mid_id:
                        mul()
                    c_id = False
                if not c_id:
                    mul(2)        # C t_l(+-), shared by the four (j, k) sign pairs
                acc(8)
    # vertices: both halves' sign products by doubling, then one accumulation
    # per vertex
    h1 = n // 2
    h2 = n - h1
    for t in range(1, h2):
        mul(2 * (1 << t))
    if not base_identity:
        mul(2)
    for t in range(1, h1):
        mul(2 * (1 << t))
    acc(1 << n)
    return c


def region_epilogue_work(unit: bool = False) -> Counter:
    """Weighting (9 generators x (basic + 4 null rules) FMA), the magnitude
    sum bounding the noise floors, the volume products, the floor tests (the
    exact floor only where the bound does not clear N_k), the error formula
    (three ratios, division each), the rounding floor of V (a 9-term FMA sum
    of |w_g| |S_g| for the positive families, a constant for the unit-bounded
    one, then two products) and the split axis."""
    c = Counter()
    floor_fma = 0 if unit else 9
    c["flops"] += 2 * 45 + 9 + 1 + 4 + 8 + 1 + 2 * floor_fma + 2
    c["inst"] += 45 + 9 + 1 + 4 + 8 + 1 + floor_fma + 2
    c["div"] += 3
    return c


def pair_table_work(family: int, n: int) -> Counter:
    """The 11-code factor table on n + 1 axes, plus the axis set-up."""
    c = Counter()
    axes = n + 1
    entries = 11 * axes
    c["flops"] += 2 * axes          # h = w/2, c = lower + h
    c["inst"] += 2 * axes
    c["flops"] += 2 * entries       # x = fma(h, g, c)
    c["inst"] += entries
    if family == PRODUCT_PEAK:
        c["flops"] += axes          # c^-2 = 1/(c c)
        c["inst"] += axes
        c["div"] += axes + entries  # and 1/(c^-2 + t^2) per entry
        c["flops"] += 3 * entries   # t = x - w, fma(t, t, c^-2)
        c["inst"] += 2 * entries
    elif family == GAUSSIAN:
        c["flops"] += 3 * entries   # x - w, a(x - w), u u
        c["inst"] += 3 * entries
        c["exp"] += entries
    elif family == C0:
        c["flops"] += 2 * entries   # x - w, a |x - w|
        c["inst"] += 2 * entries
        c["exp"] += entries
    elif family == OSCILLATORY:
        c["flops"] += entries       # a x
        c["inst"] += entries
        c["sincos"] += entries
    elif family == CORNER_PEAK:
        c["flops"] += entries       # a x
        c["inst"] += entries
    elif family == DISCONTINUOUS:
        c["flops"] += entries       # a x (the x < w test is not FP64 arithmetic)
        c["inst"] += entries
        c["exp"] += entries
    elif family == BOX_POWER:
        c["flops"] += entries       # x x
        c["inst"] += entries
    return c


def cache_fill_work(family: int, n: int, level: int) -> Counter:
    """FP64 work of filling one level of the per-axis factor cache: n 2^level
    intervals, each with the 11 entries (and set-up) of one table axis.  The
    fill kernel writes levels 0..11 once per integration."""
    one_axis = Counter(pair_table_work(family, 1))
    one_axis.subtract(pair_table_work(family, 0))
    return Counter({k: v * n * (1 << level) for k, v in one_axis.items() if v})


def pair_work(family: int, n: int, two_level: bool, cached: bool = True, q: float = 11.0) -> Counter:
    c = Counter()
    if cached:
        c["cache_loads"] += 11 * (n + 1)
    else:
        c.update(pair_table_work(family, n))
    for _ in range(2):
        c.update(region_points_work(family, n, q))
        c.update(region_epilogue_work(unit=family == 2))
        c["flops"] += 9             # two compensated adds and the rel-err test
        c["inst"] += 9
    if two_level:
        c["flops"] += 11
        c["inst"] += 8
        c["div"] += 1
    return c


def evaluate_work(family: int, n: int, regions_per_iteration, cached: bool = True, q: float = 11.0) -> Counter:
    """Total algorithmic work of the Evaluate launches of one integration,
    given the region count of every iteration (first iteration: no parents,
    no two-level refinement)."""
    tot = Counter()
    for it, s in enumerate(regions_per_iteration):
        w = pair_work(family, n, two_level=it > 0, cached=cached, q=q)
        for k, v in w.items():
            tot[k] += v * (int(s) // 2)
    return tot
