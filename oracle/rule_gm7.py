"""Genz-Malik degree-7 fully symmetric rule with its embedded degree-5 rule,
in exact rational arithmetic: the rule variant next to the degree-9 rule.

ORACLE / TEST INFRASTRUCTURE ONLY (imported by tests/ and oracle/capi.py;
never by the product package).

The paper's rule family is that of Cuhre (Sec. 2.1: the Genz-Malik rules,
2^n + Theta(n^3) points); Cuhre also offers the Genz-Malik degree-7 rule,
whose 2^n + 2n^2 + 2n + 1 points carry a degree-5 rule on all but the
vertex orbit, and whose error estimate is the difference of the two.  The
construction, written from that definition:

* five generator orbits on [-1, 1]^n: the centre; one axis at sqrt(9/70);
  one axis at sqrt(9/10); two axes at (sqrt(9/10), sqrt(9/10)); every axis
  at sqrt(9/19);
* degree-7 weights: the fully symmetric moment equations
  E[prod x_j^(2 p_j)] = prod 1/(2 p_j + 1) for every partition with
  sum p <= 3 (7 equations for n >= 3, 6 for n = 2; the radii make them
  consistent with 5 weights);
* degree-5 weights: the equations with sum p <= 2 on the first four orbits
  (the vertex orbit carries no degree-5 weight);
* error: |R7 - R5| times the region volume, i.e. the single null rule
  u = w7 - w5 (it integrates every monomial of degree <= 5 to zero);
* split axis: fourth differences from the two one-axis radii, a = sqrt(9/70)
  and b = sqrt(9/10), with q = a^2 / b^2 = 1/7.

Pinned by tests/test_oracle_rule.py: exactness of w7 on every monomial of
degree <= 7 and failure at degree 8, exactness of w5 on degree <= 5, the
point count 2^n + 2n^2 + 2n + 1.
"""
from __future__ import annotations

from decimal import Decimal
from fractions import Fraction
from functools import lru_cache

from .rule import _dsqrt, _solve_consistent, exact_moment, moment_rows, orbit_count, orbit_moment

L2 = Fraction(9, 70)
L3 = Fraction(9, 10)
L4 = Fraction(9, 10)
L5 = Fraction(9, 19)


def generator_lambdas(n: int) -> list[tuple[Fraction, ...]]:
    """Generator vectors as squared coordinates, in the fixed order: centre,
    one axis at l2, one axis at l3, two axes at l4, every axis at l5."""
    z = [Fraction(0)] * n

    def vec(*vals):
        v = list(z)
        for i, x in enumerate(vals):
            v[i] = x
        return tuple(v)

    return [vec(), vec(L2), vec(L3), vec(L4, L4), tuple([L5] * n)]


@lru_cache(maxsize=None)
def exact_rule(n: int):
    """(generators, counts, w7, w5, u = w7 - w5), exact Fractions."""
    if not 2 <= n <= 16:
        raise ValueError("dimension out of range")
    gens = generator_lambdas(n)
    cnt = [orbit_count(g) for g in gens]
    rows7 = moment_rows(n, 3)
    w7 = _solve_consistent([[orbit_moment(g, p) for g in gens] for p in rows7], [exact_moment(p) for p in rows7])
    rows5 = moment_rows(n, 2)
    w5 = _solve_consistent([[orbit_moment(g, p) for g in gens[:4]] for p in rows5],
                           [exact_moment(p) for p in rows5]) + [Fraction(0)]
    u = [a - b for a, b in zip(w7, w5)]
    return gens, cnt, w7, w5, u


def num_points(n: int) -> int:
    return sum(orbit_count(g) for g in generator_lambdas(n))


def rule_tables(n: int):
    """Double tables in the layout of oracle.rule.rule_tables: gen (G x n
    coordinate magnitudes) and wts (G x 5): column 0 the degree-7 rule,
    column 1 the null rule w7 - w5, columns 2..4 zero."""
    gens, _, w7, _, u = exact_rule(n)
    gen = [[float(_dsqrt(lam)) for lam in g] for g in gens]
    wts = [[float(Decimal(a.numerator) / Decimal(a.denominator)),
            float(Decimal(b.numerator) / Decimal(b.denominator)), 0.0, 0.0, 0.0] for a, b in zip(w7, u)]
    return gen, wts


def fourth_difference_offsets():
    """(a, b) = (sqrt(9/70), sqrt(9/10)), and q = a^2 / b^2 = 1/7."""
    return float(_dsqrt(L2)), float(_dsqrt(L3)), float(L2 / L3)
