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


# ------------------------------------------------ the degree-7 rule variant --
from oracle import rule_gm7  # noqa: E402


@pytest.mark.parametrize("n", range(2, 9))
def test_gm7_point_count_and_closed_form_weights(n):
    """2^n + 2n^2 + 2n + 1 points; the weights solved from the moment
    equations equal Genz and Malik's closed forms in n (degree 7:
    (12824 - 9120 n + 400 n^2)/19683, 980/6561, (1820 - 400 n)/19683,
    200/19683, 6859/19683/2^n; embedded degree 5: (729 - 950 n + 50 n^2)/729,
    245/486, (265 - 100 n)/1458, 25/729)."""
    assert rule_gm7.num_points(n) == 2 ** n + 2 * n * n + 2 * n + 1
    _, cnt, w7, w5, u = rule_gm7.exact_rule(n)
    F = Fraction
    assert w7 == [F(12824 - 9120 * n + 400 * n * n, 19683), F(980, 6561), F(1820 - 400 * n, 19683),
                  F(200, 19683), F(6859, 19683 * 2 ** n)]
    assert w5 == [F(729 - 950 * n + 50 * n * n, 729), F(245, 486), F(265 - 100 * n, 1458), F(25, 729), F(0)]
    assert sum(c * x for c, x in zip(cnt, w7)) == 1 and sum(c * x for c, x in zip(cnt, w5)) == 1


@pytest.mark.parametrize("n", range(2, 9))
def test_gm7_exact_for_degree_le_7_and_error_vanishes_le_5(n):
    rng = SplitMix64(177 + n)
    lo = np.array([rng.uniform(0.0, 0.5) for _ in range(n)])
    wd = np.array([rng.uniform(0.1, 0.5) for _ in range(n)])
    for p in exponent_tuples(n, 7, rng, 80):
        V, E, K, D = capi.evaluate(MONOMIAL, n, list(p), lo[None, :], wd[None, :], diag=True, degree=7)
        ex = box_monomial_integral(p, lo, lo + wd)
        assert abs(V[0] - ex) <= 1e-13 * abs(ex), (p, V[0], ex)
        if sum(p) <= 5:
            # R7 - R5 integrates degree <= 5 exactly to zero (rounding only)
            assert D[0, 0] <= 64 * rule_gm7.num_points(n) * 2.0 ** -53 * D[0, 4] + 1e-300


@pytest.mark.parametrize("n", [2, 3, 5, 8])
def test_gm7_not_exact_for_degree_8_and_error_is_the_difference(n):
    lo, wd = np.zeros(n), np.ones(n)
    p = [8] + [0] * (n - 1)
    V, E, K, D = capi.evaluate(MONOMIAL, n, p, lo[None, :], wd[None, :], diag=True, degree=7)
    assert abs(V[0] - 1 / 9) > 1e-6
    # E = |R7 - R5| for x_1^8 on [0, 1]^n, by hand: the l2 and l3 axis points
    # carry the only non-zero values off the centre, x = (1 + g)/2
    a, b = math.sqrt(9 / 70), math.sqrt(9 / 10)
    _, _, w7, w5, _ = rule_gm7.exact_rule(n)
    f = lambda g: ((1 + g) / 2) ** 8
    sums = [f(0.0), f(a) + f(-a) + (n - 1) * 2 * f(0.0), f(b) + f(-b) + (n - 1) * 2 * f(0.0)]
    pair = 2 * (n - 1) * (f(b) + f(-b)) + 4 * (n - 1) * (n - 2) // 2 * f(0.0)
    vert = 2 ** (n - 1) * (f(math.sqrt(9 / 19)) + f(-math.sqrt(9 / 19)))
    S = sums + [pair, vert]
    r7 = sum(float(w) * s for w, s in zip(w7, S))
    r5 = sum(float(w) * s for w, s in zip(w5, S))
    assert abs(V[0] - r7) <= 1e-14
    assert abs(E[0] - abs(r7 - r5)) <= 1e-14


def test_gm7_split_axis_uses_its_radii():
    # f = x_0^4 on [0,1]^2: D_0 = 2 a^2 h^4 |a^2 - b^2| with a^2 = 9/70,
    # b^2 = 9/10, h = 1/2 (second differences 12 c^2 r^2 h^2 + 2 r^4 h^4)
    V, E, K, D = capi.evaluate(MONOMIAL, 2, [4, 0], [[0.0, 0.0]], [[1.0, 1.0]], diag=True, degree=7)
    a2, b2, h = 9 / 70, 9 / 10, 0.5
    assert abs(D[0, 9] - 2 * a2 * h ** 4 * abs(a2 - b2)) < 1e-16
    assert D[0, 10] == 0.0 and K[0] == 0
