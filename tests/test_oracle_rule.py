"""Pins of the oracle's cubature rule (oracle/rule.py) and of the orbit
enumeration and affine map in the C oracle (oracle/pagani_oracle.c).

The paper fixes the rule family: Genz-Malik / DCUHRE degree 9 with
2^n + Theta(n^3) points (Sec. 2.1) and four null rules (Sec. 3.2).  Checked
here against mathematics that does not come from the oracle itself: exact
integrals of monomials over boxes, the closed-form point count, annihilation
of low-degree monomials by the null rules, orthogonality and equal norms.
"""
import itertools
import math
from decimal import Decimal
from fractions import Fraction

import numpy as np
import pytest

from oracle import capi, rule
from paper_2104_06494_gb300.workloads import SplitMix64

MONOMIAL = 100


def count_formula(n):
    return 1 + 8 * n + 6 * n * (n - 1) + 4 * n * (n - 1) * (n - 2) // 3 + 2 ** n


@pytest.mark.parametrize("n", range(2, 9))
def test_point_count(n):
    assert rule.num_points(n) == count_formula(n)


def test_point_count_values():
    assert [rule.num_points(n) for n in (3, 5, 6, 8)] == [77, 273, 453, 1105]


@pytest.mark.parametrize("n", range(2, 9))
def test_weights_normalised(n):
    gens, cnt, w, _, _ = rule.exact_rule(n)
    assert sum(c * x for c, x in zip(cnt, w)) == 1
    # the lambda_p generator carries zero basic weight (it serves the null
    # rules and the fourth difference only)
    assert w[4] == 0


def box_monomial_integral(p, lo, hi):
    out = 1.0
    for e, a, b in zip(p, lo, hi):
        out *= (b ** (e + 1) - a ** (e + 1)) / (e + 1)
    return out


def exponent_tuples(n, maxdeg, rng, limit):
    allp = [p for p in itertools.product(range(maxdeg + 1), repeat=n) if sum(p) <= maxdeg]
    if len(allp) <= limit:
        return allp
    idx = sorted({int(rng.uniform(0, len(allp))) for _ in range(limit)})
    return [allp[i] for i in idx]


@pytest.mark.parametrize("n", range(2, 9))
def test_exact_for_degree_le_9(n):
    rng = SplitMix64(77 + n)
    lo = np.array([rng.uniform(0.0, 0.5) for _ in range(n)])
    wd = np.array([rng.uniform(0.1, 0.5) for _ in range(n)])
    ps = exponent_tuples(n, 9, rng, 120)
    for p in ps:
        V, E, K = capi.evaluate(MONOMIAL, n, list(p), lo[None, :], wd[None, :])
        ex = box_monomial_integral(p, lo, lo + wd)
        assert abs(V[0] - ex) <= 1e-13 * abs(ex), (p, V[0], ex)


@pytest.mark.parametrize("n", [2, 3, 5, 8])
def test_not_exact_for_degree_10(n):
    lo = np.zeros(n)
    wd = np.ones(n)
    p = [10] + [0] * (n - 1)
    V, _, _ = capi.evaluate(MONOMIAL, n, p, lo[None, :], wd[None, :])
    assert abs(V[0] - 1 / 11) > 1e-8


@pytest.mark.parametrize("n", [2, 3, 4, 6, 8])
def test_null_rules_annihilate(n):
    """u_k annihilates every monomial (symmetric or not) of degree <= delta_k
    and fails on x_1^(delta_k + 1)."""
    rng = SplitMix64(500 + n)
    lo = np.array([rng.uniform(0.0, 0.5) for _ in range(n)])
    wd = np.array([rng.uniform(0.1, 0.5) for _ in range(n)])
    for k, deg in enumerate(rule.NULL_DEGREES):
        for p in exponent_tuples(n, deg, rng, 60):
            _, _, _, D = capi.evaluate(MONOMIAL, n, list(p), lo[None, :], wd[None, :], diag=True)
            assert D[0, k] <= 1e-13 * D[0, 4 + k], (k, p, D[0, k], D[0, 4 + k])
        p = [deg + 1] + [0] * (n - 1)
        _, _, _, D = capi.evaluate(MONOMIAL, n, p, np.zeros((1, n)), np.ones((1, n)), diag=True)
        assert D[0, k] > 1e-9 * D[0, 4 + k], (k, p)


@pytest.mark.parametrize("n", range(2, 9))
def test_null_rules_orthogonal_equal_norm(n):
    gens, cnt, w, nulls_exact, nulls = rule.exact_rule(n)
    for i in range(4):
        for j in range(i):
            assert sum(c * a * b for c, a, b in zip(cnt, nulls_exact[i], nulls_exact[j])) == 0
    wn = sum(c * x * x for c, x in zip(cnt, w))
    wn = Decimal(wn.numerator) / Decimal(wn.denominator)
    for u in nulls:
        un = sum(Decimal(c) * x * x for c, x in zip(cnt, u))
        assert abs(un / wn - 1) < Decimal("1e-40")
    assert all(any(x != 0 for x in u) for u in nulls_exact)


@pytest.mark.parametrize("n", [2, 5, 8])
def test_tables_round_correctly(n):
    gen, wts = rule.rule_tables(n)
    gens, cnt, w, _, nulls = rule.exact_rule(n)
    for g in range(len(gens)):
        assert wts[g][0] == float(Fraction(w[g]))
        for j in range(n):
            assert abs(gen[g][j] ** 2 - float(gens[g][j])) <= 4e-16 * max(1.0, float(gens[g][j]))


def test_lambdas_match_construction():
    lam = {k: float(v) for k, v in rule.lambdas().items()}
    assert lam["l0"] == 0.4707 and lam["lp"] == 0.0625
    assert abs(lam["l1"] - 4 / (15 - 5 / 0.4707)) < 1e-15
    # every generator radius lies inside the reference cube
    assert all(0 < v < 1 for v in lam.values())
