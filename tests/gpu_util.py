"""Helpers shared by the GPU parity tests: tolerances derived from the
floating-point arithmetic, the reference error formula applied to given
null-rule values, and the comparison of two integration runs."""
import math

import numpy as np

EPS = 2.0 ** -53


def point_count(n):
    return 1 + 8 * n + 6 * n * (n - 1) + 4 * n * (n - 1) * (n - 2) // 3 + 2 ** n


def value_condition(family, n, params, lo, wd):
    """Per-box rounding sensitivity of the integrand values: (k_rel, k_abs)
    such that one evaluation of f at a point of the box carries an error of
    at most k_rel eps |f| + k_abs eps, whichever way it is formed (products
    of per-axis factors or the formula written out):
      product peak  k_rel = 2n + 4 (n divisions and products)
      Gaussian      k_rel = max sum (3 u^2 + 2 |u| |a| |x|) + n + 4, u = a (x - w)
                    (exp turns an absolute error of its argument into a
                    relative error of its value; the point coordinate x
                    carries eps |x|, which u^2 turns into 2 |u| |a| eps |x|)
      C0            k_rel = max sum (2 |u| + |a| |x|) + n + 4, u = a |x - w|
      corner peak   k_rel = 4 (n + 1) (a power of a sum of n terms)
      oscillatory   k_abs = 2 pi |u| + sum |a| max |x| (the cosine argument)
      discontinuous k_rel = 2n + 4 + max sum |a x| (the exponent)
      box power     k_rel = q (n + 2 + 2 (1 + hi / x_min)) + 8: a point
                    coordinate x = c + h g carries an absolute error of
                    about eps hi, relative 1 + hi / x at its smallest x
                    (the largest generator radius 0.956 leaves
                    x_min >= lo + 0.022 w), squared, summed over n axes and
                    raised to the power q"""
    lo = np.atleast_2d(lo)
    hi = lo + np.atleast_2d(wd)
    m = lo.shape[0]
    p = np.asarray(params, dtype=np.float64)
    k_rel = np.full(m, 2.0 * n + 4)
    k_abs = np.zeros(m)
    xmax = np.maximum(np.abs(lo), np.abs(hi))
    if family == 1:
        a, w = p[:n], p[n:]
        u = np.abs(a) * np.maximum(np.abs(lo - w), np.abs(hi - w))
        k_rel = np.sum(3 * u ** 2 + 2 * u * np.abs(a) * xmax, axis=1) + n + 4
    elif family == 4:
        a, w = p[:n], p[n:]
        u = np.abs(a) * np.maximum(np.abs(lo - w), np.abs(hi - w))
        k_rel = np.sum(2 * u + np.abs(a) * xmax, axis=1) + n + 4
    elif family == 3:
        k_rel = np.full(m, 4.0 * (n + 1))
    elif family == 2:
        k_abs = 2 * np.pi * abs(p[0]) + np.sum(np.abs(p[1:]) * np.maximum(np.abs(lo), np.abs(hi)), axis=1)
    elif family == 5:
        a = p[:n]
        k_rel = 2.0 * n + 4 + np.sum(np.abs(a) * np.maximum(np.abs(lo), np.abs(hi)), axis=1)
    elif family == 6:
        q = abs(p[0])
        xmin = lo + 0.022 * (hi - lo)
        k_rel = q * (n + 2 + 2 * (1 + np.max(hi / xmin, axis=1))) + 8
    return k_rel, k_abs


def sum_tolerance(n, scale, k_rel=0.0, abs_scale=0.0, k_abs=0.0):
    """Bound on the difference of two evaluations of a weighted sum of the
    N(n) integrand values of a box computed in different orders and ways:
    (N + 2n + 16 + k_rel) eps sum |w f| + k_abs eps sum |w| vol (recursive
    summation bound plus the per-value error of value_condition)."""
    return (point_count(n) + 2 * n + 16 + k_rel) * EPS * scale + k_abs * EPS * abs_scale


def null_error(n1, n2, n3, n4):
    """Region error from four null values, the reading of Sec. 3.2 used by
    both implementations (restated here to check the kernel's epilogue
    against its own N_k); the rounding floor of V is applied on top."""
    def ratio(x, y):
        return x / y if y > 0 else (math.inf if x > 0 else 0.0)
    r = max(ratio(n1, n2), ratio(n2, n3), ratio(n3, n4))
    if r >= 1:
        return 10 * max(n1, n2, n3)
    return 10 * r * max(n1, r * n2)


# no region error below 16 u times the rule's absolute sum of V
V_ROUND = 16 * 2.0 ** -53


def sibling_regions(n, m, seed, max_level=10):
    """m regions forming sibling pairs (2i, 2i+1): halves of random dyadic
    parents along random axes; returned as (m x n) lower, width lists."""
    from paper_2104_06494_gb300.workloads import SplitMix64
    rng = SplitMix64(seed)
    lo, wd = [], []
    while len(lo) < m:
        plo, pwd = [], []
        for _ in range(n):
            lvl = int(rng.uniform(0, max_level + 1))
            k = int(rng.uniform(0, 1 << lvl))
            plo.append(k / (1 << lvl))
            pwd.append(1.0 / (1 << lvl))
        ax = int(rng.uniform(0, n))
        a, b = list(plo), list(pwd)
        b[ax] = pwd[ax] / 2
        c, d = list(plo), list(b)
        c[ax] = plo[ax] + b[ax]
        lo += [a, c]
        wd += [b, d]
    return np.array(lo[:m]), np.array(wd[:m])


def close(a, b, rel=1e-12, floor=1e-300):
    return abs(a - b) <= rel * max(abs(a), abs(b)) + floor


def compare_runs(g, o, rel=1e-12, value_scale=0.0):
    """Equal region sets (statuses, iterations, per-iteration counts and
    decisions), integral estimates within 1e-12 relative.  Error estimates are
    sums of region errors computed from null-rule values, differences of
    nearly equal sums known only to their rounding level; they are compared
    to 1e-6 relative, or 1e-12 of the integral's magnitude where they are
    themselves at that noise level.  value_scale: the integral of |f| where
    it exceeds |I| (a sign-changing integrand cancels: its sums carry
    rounding errors relative to the integral of |f|, 1 for |f| <= 1 on the
    unit cube, not to the small integral itself)."""
    assert g.status == o.status, (g.status, o.status)
    assert g.iterations == o.iterations
    assert g.n_regions == o.n_regions
    assert g.n_active_last == o.n_active_last
    scale = max(abs(o.estimate), float(np.max(np.abs(o.trace["v"]) + np.abs(o.trace["vf"]))), value_scale)
    assert abs(g.estimate - o.estimate) <= rel * scale + 1e-300, (g.estimate, o.estimate)
    efloor = 1e-12 * scale
    assert close(g.errorest, o.errorest, rel=1e-6, floor=efloor), (g.errorest, o.errorest)
    gt, ot = g.trace, o.trace
    assert len(gt) == len(ot)
    for a, b in zip(gt, ot):
        for key in ("it", "trigger", "probes", "search_ok", "s", "n_relerr_active", "n_survivors"):
            assert a[key] == b[key], (key, a, b)
        assert abs(a["v"] - b["v"]) <= rel * scale
        assert abs(a["vf"] - b["vf"]) <= rel * scale
        assert close(a["e"], b["e"], rel=1e-6, floor=efloor), (a["e"], b["e"])
        assert close(a["ef"], b["ef"], rel=1e-6, floor=efloor), (a["ef"], b["ef"])
