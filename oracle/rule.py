"""Degree-9 fully symmetric cubature rule and its four null rules, in exact
rational arithmetic.

ORACLE / TEST INFRASTRUCTURE ONLY.  Nothing in the product package may import
this module; only tests/, the smoke check and the CPU baseline of bench.py use it.

What the paper fixes (Sec. 2.1 "Cuba: Cuhre", Sec. 3.2 "Region Evaluation"):
the rule family is the Genz-Malik / DCUHRE degree-9 rule with 2^n + Theta(n^3)
points, and four further rules give four estimates whose largest difference
yields the region error.  The paper prints neither the generators, the weights
nor the null rules.  The reading used here:

* Generators (squared radii, lambda):  l0 = 0.4707,
  l1 = 4/(15 - 5/l0),  rho = (1 - l1/l0)/27,
  l2 = (5 - 7 l1 - 35 rho)/(7 - 35 l1/3 - 35 rho/l0),
  rho' = rho (1 - l2/l0)/3,
  l3 = (7 - 9(l2+l1) + 63 l2 l1/5 - 63 rho')/(9 - 63(l2+l1)/5 + 21 l2 l1 - 63 rho'/l0),
  lp = 1/16.
  Every lambda is rational because l0 is, so the whole construction is exact.
* Nine generator orbits on [-1,1]^n (all distinct coordinate permutations and
  all sign changes of the generator vector): the centre; one axis at sqrt(l1),
  sqrt(l2), sqrt(l3), sqrt(lp); two axes at (sqrt(l1), sqrt(l1)); two axes at
  (sqrt(l1), sqrt(l2)); three axes at sqrt(l1); every axis at sqrt(l0).
* Basic weights: the fully symmetric moment equations
  E[prod x_j^(2 p_j)] = prod 1/(2 p_j + 1) for every partition with sum p <= 4
  (normalised so that the weights of all points sum to 1).
* Null rule u_k (k = 1..4) of degree delta_k = 7, 5, 3, 1: the projection of
  the basic weight vector onto the null space of the moment equations of
  degree <= delta_k, in the inner product <a, b> = sum_g count_g a_g b_g,
  made orthogonal to u_1..u_{k-1}, then scaled to the norm of the basic rule.

Pinned by tests/test_oracle_rule.py: exactness on every monomial of degree
<= 9 and failure on degree 10, annihilation of every monomial of degree
<= delta_k by u_k, mutual orthogonality, equal norms, point counts.
"""
from __future__ import annotations

import itertools
from decimal import Decimal, getcontext
from fractions import Fraction
from functools import lru_cache

getcontext().prec = 60

# ---------------------------------------------------------------- lambdas --
L0 = Fraction(4707, 10000)
L1 = 4 / (15 - 5 / L0)
_RHO = (1 - L1 / L0) / 27
L2 = (5 - 7 * L1 - 35 * _RHO) / (7 - Fraction(35, 3) * L1 - 35 * _RHO / L0)
_RHO2 = _RHO * (1 - L2 / L0) / 3
L3 = (7 - 9 * (L2 + L1) + Fraction(63, 5) * L2 * L1 - 63 * _RHO2) / (
    9 - Fraction(63, 5) * (L2 + L1) + 21 * L2 * L1 - 63 * _RHO2 / L0)
LP = Fraction(1, 16)

NULL_DEGREES = (7, 5, 3, 1)


def generator_lambdas(n: int) -> list[tuple[Fraction, ...]]:
    """Generator vectors as squared coordinates (length n, zeros padded), in
    the fixed order used everywhere in the oracle."""
    z = [Fraction(0)] * n

    def vec(*vals):
        v = list(z)
        for i, x in enumerate(vals):
            v[i] = x
        return tuple(v)

    gens = [vec(), vec(L1), vec(L2), vec(L3), vec(LP), vec(L1, L1), vec(L1, L2)]
    if n >= 3:
        gens.append(vec(L1, L1, L1))
    gens.append(tuple([L0] * n))
    return gens


GENERATOR_NAMES_3 = ["centre", "l1", "l2", "l3", "lp", "l1l1", "l1l2", "l1l1l1", "l0^n"]


def generator_names(n: int) -> list[str]:
    names = list(GENERATOR_NAMES_3)
    if n < 3:
        names.remove("l1l1l1")
    return names


@lru_cache(maxsize=None)
def orbit_lambda_points(gen: tuple[Fraction, ...]) -> tuple[tuple[tuple[Fraction, ...], int], ...]:
    """Distinct coordinate permutations of a generator (as squared values)
    with the number of sign patterns each carries (2^#nonzero)."""
    perms = set(itertools.permutations(gen))
    nz = sum(1 for x in gen if x != 0)
    return tuple((p, 2 ** nz) for p in sorted(perms))


def orbit_count(gen) -> int:
    return sum(m for _, m in orbit_lambda_points(tuple(gen)))


def partitions(k: int, maxparts: int, maxpart: int | None = None):
    """Partitions of k into at most maxparts positive parts, non-increasing."""
    if maxpart is None:
        maxpart = k
    if k == 0:
        yield ()
        return
    if maxparts == 0:
        return
    for first in range(min(k, maxpart), 0, -1):
        for rest in partitions(k - first, maxparts - 1, first):
            yield (first,) + rest


def moment_rows(n: int, max_half_degree: int):
    """All fully symmetric moment conditions with sum(p) <= max_half_degree."""
    rows = []
    for k in range(max_half_degree + 1):
        rows.extend(partitions(k, n))
    return rows


def orbit_moment(gen, p) -> Fraction:
    """sum over the orbit of gen of prod_j x_j^(2 p_j) (p padded with zeros)."""
    n = len(gen)
    pp = tuple(p) + (0,) * (n - len(p))
    total = Fraction(0)
    for pt, mult in orbit_lambda_points(tuple(gen)):
        term = Fraction(1)
        for lam, e in zip(pt, pp):
            if e:
                term *= lam ** e
        total += mult * term
    return total


def exact_moment(p) -> Fraction:
    out = Fraction(1)
    for e in p:
        out /= (2 * e + 1)
    return out


def _solve_consistent(rows: list[list[Fraction]], rhs: list[Fraction]) -> list[Fraction]:
    """Exact Gauss-Jordan on an overdetermined system; raises if inconsistent
    or if the solution is not unique."""
    m = len(rows)
    ncol = len(rows[0])
    a = [list(r) + [b] for r, b in zip(rows, rhs)]
    piv_cols = []
    r = 0
    for c in range(ncol):
        piv = next((i for i in range(r, m) if a[i][c] != 0), None)
        if piv is None:
            continue
        a[r], a[piv] = a[piv], a[r]
        inv = 1 / a[r][c]
        a[r] = [x * inv for x in a[r]]
        for i in range(m):
            if i != r and a[i][c] != 0:
                f = a[i][c]
                a[i] = [x - f * y for x, y in zip(a[i], a[r])]
        piv_cols.append(c)
        r += 1
    for i in range(r, m):
        if a[i][ncol] != 0:
            raise ValueError("moment equations are inconsistent")
    if r != ncol:
        raise ValueError("moment equations do not fix the weights")
    return [a[i][ncol] for i in range(ncol)]


def _nullspace_projector_apply(S: list[list[Fraction]], cnt: list[int], x: list[Fraction]) -> list[Fraction]:
    """Project x onto {a : sum_g a_g S[r][g] = 0 for all rows r} orthogonally
    in the inner product <a,b> = sum_g cnt_g a_g b_g."""
    # P x = x - Minv S^T (S Minv S^T)^+ S x ; rows of S may be dependent, so
    # first reduce S to an independent row set.
    G = len(x)
    basis = []
    for row in S:
        cand = list(row)
        # test independence by exact elimination against the basis
        trial = basis + [cand]
        if _rank(trial) == len(trial):
            basis.append(cand)
    if not basis:
        return list(x)
    minv = [Fraction(1, c) for c in cnt]
    k = len(basis)
    gram = [[sum(basis[i][g] * minv[g] * basis[j][g] for g in range(G)) for j in range(k)] for i in range(k)]
    sx = [sum(basis[i][g] * x[g] for g in range(G)) for i in range(k)]
    y = _solve_consistent(gram, sx)
    return [x[g] - minv[g] * sum(basis[i][g] * y[i] for i in range(k)) for g in range(G)]


def _rank(rows: list[list[Fraction]]) -> int:
    a = [list(r) for r in rows]
    m, ncol = len(a), len(a[0])
    r = 0
    for c in range(ncol):
        piv = next((i for i in range(r, m) if a[i][c] != 0), None)
        if piv is None:
            continue
        a[r], a[piv] = a[piv], a[r]
        for i in range(r + 1, m):
            if a[i][c] != 0:
                f = a[i][c] / a[r][c]
                a[i] = [x - f * y for x, y in zip(a[i], a[r])]
        r += 1
    return r


def _inner(a, b, cnt) -> Fraction:
    return sum(c * x * y for c, x, y in zip(cnt, a, b))


def _dsqrt(q: Fraction) -> Decimal:
    return (Decimal(q.numerator) / Decimal(q.denominator)).sqrt()


@lru_cache(maxsize=None)
def exact_rule(n: int):
    """Returns (generators, counts, basic weights w, null rules u_1..u_4 as
    Decimal vectors).  The basic weights are exact Fractions; the null rules
    carry one square root each and are returned at 60 significant digits."""
    if not 2 <= n <= 16:
        raise ValueError("dimension out of range")
    gens = generator_lambdas(n)
    cnt = [orbit_count(g) for g in gens]
    prts = moment_rows(n, 4)
    S = [[orbit_moment(g, p) for g in gens] for p in prts]
    w = _solve_consistent(S, [exact_moment(p) for p in prts])
    nulls_exact = []
    for deg in NULL_DEGREES:
        rows = [[orbit_moment(g, p) for g in gens] for p in moment_rows(n, (deg - 1) // 2)]
        u = _nullspace_projector_apply(rows, cnt, w)
        for prev in nulls_exact:
            c = _inner(u, prev, cnt) / _inner(prev, prev, cnt)
            u = [x - c * y for x, y in zip(u, prev)]
        nulls_exact.append(u)
    wnorm2 = _inner(w, w, cnt)
    nulls = []
    for u in nulls_exact:
        scale = _dsqrt(wnorm2 / _inner(u, u, cnt))
        nulls.append([Decimal(x.numerator) / Decimal(x.denominator) * scale for x in u])
    return gens, cnt, w, nulls_exact, nulls


def num_points(n: int) -> int:
    return sum(orbit_count(g) for g in generator_lambdas(n))


def rule_tables(n: int):
    """Double-precision tables for the C oracle.

    Returns (gen, wts): gen is G x n coordinate magnitudes sqrt(lambda)
    (correctly rounded from 60-digit decimals), wts is G x 5 with column 0 the
    basic rule and columns 1..4 the null rules u_1..u_4 (all normalised to the
    unit-volume reference cube; the region volume multiplies them)."""
    gens, cnt, w, _, nulls = exact_rule(n)
    gen = [[float(_dsqrt(lam)) for lam in g] for g in gens]
    wts = []
    for gi in range(len(gens)):
        row = [float(Decimal(w[gi].numerator) / Decimal(w[gi].denominator))]
        row += [float(nulls[k][gi]) for k in range(4)]
        wts.append(row)
    return gen, wts


def fourth_difference_offsets(outer: bool = True):
    """(a, b): the two one-axis radii whose second differences are combined
    into a fourth difference, with weight q = a^2 / b^2
    (fourth_difference_weight).  outer: the inner and the outer radius of the
    rule, (sqrt(l2), sqrt(l1)), as Genz and Malik's rule takes its difference
    at its inner and outer radii sqrt(9/70) and sqrt(9/10); used for the
    smooth families.  Otherwise the two inner radii (sqrt(lp), sqrt(l2)),
    used for the families with kinks or jumps, where a difference reaching
    out to sqrt(l1) bisects boxes across features that then sit in the
    children's outer margin, beyond every rule point."""
    if outer:
        return float(_dsqrt(L2)), float(_dsqrt(L1))
    return float(_dsqrt(LP)), float(_dsqrt(L2))


def fourth_difference_weight(outer: bool = True) -> Fraction:
    """q = a^2 / b^2: l2 / l1 (outer), lp / l2 (inner)."""
    return L2 / L1 if outer else LP / L2


def lambdas():
    return {"l0": L0, "l1": L1, "l2": L2, "l3": L3, "lp": LP}
