"""Closed-form integrals over [0,1]^n of the five synthetic integrand families.

ORACLE / TEST INFRASTRUCTURE ONLY (imported by tests/, the smoke check and the
CPU baseline of bench.py; never by the product package).

The paper argues for Genz families with fixed parameters so that analytic
values exist (Sec. 4.2 "Accuracy"); it prints the formulas (Sec. 4.1) but no
values.  These are the integrals written out, one 1-D factor per axis where
the family is a product:

* product peak  prod_j 1/(c_j^-2 + (x_j - w_j)^2):
      prod_j c_j [atan(c_j (1 - w_j)) + atan(c_j w_j)]
* Gaussian      exp(-sum_j a_j^2 (x_j - w_j)^2):
      prod_j sqrt(pi)/(2 a_j) [erf(a_j (1 - w_j)) + erf(a_j w_j)]
* oscillatory   cos(2 pi u + sum_j a_j x_j):
      Re[ exp(2 pi i u) prod_j (exp(i a_j) - 1)/(i a_j) ]
* corner peak   (1 + sum_j a_j x_j)^-(n+1):
      1/(n! prod_j a_j) sum_{S subset [n]} (-1)^|S| / (1 + sum_{j in S} a_j)
  evaluated in exact rational arithmetic (the alternating sum cancels heavily)
* C0            exp(-sum_j a_j |x_j - w_j|):
      prod_j (2 - exp(-a_j w_j) - exp(-a_j (1 - w_j))) / a_j
* discontinuous exp(sum_j a_j x_j) if every x_j < w_j, else 0 (paper f6):
      prod_j (exp(a_j min(w_j, 1)) - 1) / a_j
* box power     (sum_j x_j^2)^q (paper f7, f8): for integer q the multinomial
      expansion sum_{k_1+..+k_n=q} q!/prod k_j! prod 1/(2 k_j + 1), exact
      rationals; no closed form for other q (None)

closed_form_box gives the same integrals over a general box [lo, hi].

Pinned in tests/test_oracle_closed_forms.py against tensor Gauss-Legendre
quadrature (split at the kink for C0) in low dimension.
"""
from __future__ import annotations

import cmath
import itertools
import math
from fractions import Fraction

PRODUCT_PEAK, GAUSSIAN, OSCILLATORY, CORNER_PEAK, C0, DISCONTINUOUS, BOX_POWER = 0, 1, 2, 3, 4, 5, 6


def closed_form(family: int, n: int, params) -> float:
    p = [float(x) for x in params]
    if family == PRODUCT_PEAK:
        c, w = p[:n], p[n:2 * n]
        return math.prod(cj * (math.atan(cj * (1 - wj)) + math.atan(cj * wj)) for cj, wj in zip(c, w))
    if family == GAUSSIAN:
        a, w = p[:n], p[n:2 * n]
        return math.prod(math.sqrt(math.pi) / (2 * aj) * (math.erf(aj * (1 - wj)) + math.erf(aj * wj))
                         for aj, wj in zip(a, w))
    if family == OSCILLATORY:
        u, a = p[0], p[1:1 + n]
        z = cmath.exp(2j * math.pi * u)
        for aj in a:
            z *= (cmath.exp(1j * aj) - 1) / (1j * aj)
        return z.real
    if family == CORNER_PEAK:
        a = [Fraction(x) for x in p[:n]]
        tot = Fraction(0)
        for k in range(n + 1):
            for S in itertools.combinations(range(n), k):
                tot += Fraction((-1) ** k) / (1 + sum((a[j] for j in S), Fraction(0)))
        return float(tot / (math.factorial(n) * math.prod(a)))
    if family == C0:
        a, w = p[:n], p[n:2 * n]
        return math.prod((2 - math.exp(-aj * wj) - math.exp(-aj * (1 - wj))) / aj for aj, wj in zip(a, w))
    if family == DISCONTINUOUS:
        a, w = p[:n], p[n:2 * n]
        out = 1.0
        for aj, wj in zip(a, w):
            hi = min(max(wj, 0.0), 1.0)
            out *= math.expm1(aj * hi) / aj
        return out
    if family == BOX_POWER:
        q = p[0]
        if q != int(q) or q < 0:
            return None
        q = int(q)
        tot = Fraction(0)
        for ks in _compositions(q, n):
            term = Fraction(math.factorial(q))
            for k in ks:
                term /= math.factorial(k) * (2 * k + 1)
            tot += term
        return float(tot)
    raise ValueError(f"unknown family {family}")


def closed_form_box(family: int, n: int, params, lo, hi) -> float:
    """The integral over the box [lo, hi] (Algorithm 2's bounds a, b), one
    1-D antiderivative per axis for the product families:
      product peak  c [atan(c (hi - w)) - atan(c (lo - w))]
      Gaussian      sqrt(pi)/(2 a) [erf(a (hi - w)) - erf(a (lo - w))] (via
                    erfc when both ends lie on one side of w, against
                    cancellation)
      oscillatory   Re[exp(2 pi i u) prod (exp(i a hi) - exp(i a lo))/(i a)]
      C0            the kink at w splits the axis into up to two exponentials
      discontinuous (exp(a min(hi, w)) - exp(a lo))/a, or 0 when w <= lo
    the corner peak as the signed vertex sum 1/(n! prod a) sum_v
    (-1)^{#v_j = hi_j} / (1 + a.v) (n integrations of (1 + a.x)^-(k+1)), in
    exact rationals; the integer box power as the multinomial sum of
    prod (hi^(2k+1) - lo^(2k+1))/(2k+1), exact."""
    p = [float(x) for x in params]
    lo = [float(x) for x in lo]
    hi = [float(x) for x in hi]
    if family == PRODUCT_PEAK:
        c, w = p[:n], p[n:2 * n]
        return math.prod(cj * (math.atan(cj * (h - wj)) - math.atan(cj * (l - wj)))
                         for cj, wj, l, h in zip(c, w, lo, hi))
    if family == GAUSSIAN:
        a, w = p[:n], p[n:2 * n]
        out = 1.0
        for aj, wj, l, h in zip(a, w, lo, hi):
            x0, x1 = aj * (l - wj), aj * (h - wj)
            if x0 >= 0:
                d = math.erfc(x0) - math.erfc(x1)
            elif x1 <= 0:
                d = math.erfc(-x1) - math.erfc(-x0)
            else:
                d = math.erf(x1) - math.erf(x0)
            out *= math.sqrt(math.pi) / (2 * aj) * d
        return out
    if family == OSCILLATORY:
        u, a = p[0], p[1:1 + n]
        z = cmath.exp(2j * math.pi * u)
        for aj, l, h in zip(a, lo, hi):
            z *= (cmath.exp(1j * aj * h) - cmath.exp(1j * aj * l)) / (1j * aj)
        return z.real
    if family == CORNER_PEAK:
        a = [Fraction(x) for x in p[:n]]
        L = [Fraction(x) for x in lo]
        H = [Fraction(x) for x in hi]
        tot = Fraction(0)
        for v in itertools.product((0, 1), repeat=n):
            pt = [H[j] if v[j] else L[j] for j in range(n)]
            tot += Fraction((-1) ** sum(v)) / (1 + sum((a[j] * pt[j] for j in range(n)), Fraction(0)))
        return float(tot / (math.factorial(n) * math.prod(a)))
    if family == C0:
        a, w = p[:n], p[n:2 * n]
        out = 1.0
        for aj, wj, l, h in zip(a, w, lo, hi):
            if h <= wj:
                f = (math.exp(-aj * (wj - h)) - math.exp(-aj * (wj - l))) / aj
            elif l >= wj:
                f = (math.exp(-aj * (l - wj)) - math.exp(-aj * (h - wj))) / aj
            else:
                f = (2 - math.exp(-aj * (wj - l)) - math.exp(-aj * (h - wj))) / aj
            out *= f
        return out
    if family == DISCONTINUOUS:
        a, w = p[:n], p[n:2 * n]
        out = 1.0
        for aj, wj, l, h in zip(a, w, lo, hi):
            top = min(h, wj)
            if top <= l:
                return 0.0
            out *= math.exp(aj * l) * math.expm1(aj * (top - l)) / aj
        return out
    if family == BOX_POWER:
        q = p[0]
        if q != int(q) or q < 0:
            return None
        q = int(q)
        L = [Fraction(x) for x in lo]
        H = [Fraction(x) for x in hi]
        tot = Fraction(0)
        for ks in _compositions(q, n):
            term = Fraction(math.factorial(q))
            for j, k in enumerate(ks):
                term *= (H[j] ** (2 * k + 1) - L[j] ** (2 * k + 1)) / (math.factorial(k) * (2 * k + 1))
            tot += term
        return float(tot)
    raise ValueError(f"unknown family {family}")


def _compositions(total: int, parts: int):
    """All (k_1..k_parts) of non-negative integers summing to total."""
    if parts == 1:
        yield (total,)
        return
    for first in range(total + 1):
        for rest in _compositions(total - first, parts - 1):
            yield (first,) + rest


def gaussian_gradient(n: int, params):
    """d/d(a, w) of the Gaussian family's closed form: with the 1-D factor
    F_j = sqrt(pi)/(2 a) [erf(a (1 - w)) + erf(a w)],
    dF_j/dw = exp(-a^2 w^2) - exp(-a^2 (1 - w)^2) and
    dF_j/da = -F_j / a + [(1 - w) exp(-a^2 (1 - w)^2) + w exp(-a^2 w^2)] / a."""
    p = [float(x) for x in params]
    a, w = p[:n], p[n:2 * n]
    F = [math.sqrt(math.pi) / (2 * aj) * (math.erf(aj * (1 - wj)) + math.erf(aj * wj)) for aj, wj in zip(a, w)]
    tot = math.prod(F)
    ga, gw = [], []
    for j, (aj, wj) in enumerate(zip(a, w)):
        rest = math.prod(F[:j] + F[j + 1:])
        dw = math.exp(-aj * aj * wj * wj) - math.exp(-aj * aj * (1 - wj) ** 2)
        da = -F[j] / aj + ((1 - wj) * math.exp(-aj * aj * (1 - wj) ** 2) + wj * math.exp(-aj * aj * wj * wj)) / aj
        ga.append(da * rest)
        gw.append(dw * rest)
    return tot, ga + gw
