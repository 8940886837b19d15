"""Pins of oracle/closed_forms.py against brute-force composite tensor
Gauss-Legendre quadrature in 2-D and 3-D (panels split at w for the C0 kink
and the discontinuous family's jump), of the corner-peak formula against its
1-D antiderivative, and of the oracle's whole integration of the box power
with a non-integer exponent (paper f8, no closed form) against quadrature."""
import json
import math
import os

import numpy as np
import pytest

from oracle import closed_forms as cf
from oracle import capi
from paper_2104_06494_gb300.workloads import (draw_params, PRODUCT_PEAK, GAUSSIAN, OSCILLATORY, CORNER_PEAK, C0,
                                            DISCONTINUOUS, BOX_POWER)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def f_numpy(family, n, p, X):
    """Integrand on an array of points X (m x n), written from the formulas."""
    p = np.asarray(p, dtype=np.float64)
    if family == PRODUCT_PEAK:
        c, w = p[:n], p[n:]
        return np.prod(1.0 / (c ** -2.0 + (X - w) ** 2), axis=1)
    if family == GAUSSIAN:
        a, w = p[:n], p[n:]
        return np.exp(-np.sum(a ** 2 * (X - w) ** 2, axis=1))
    if family == OSCILLATORY:
        return np.cos(2 * np.pi * p[0] + X @ p[1:])
    if family == CORNER_PEAK:
        return (1.0 + X @ p) ** (-(n + 1))
    if family == C0:
        a, w = p[:n], p[n:]
        return np.exp(-np.sum(a * np.abs(X - w), axis=1))
    if family == DISCONTINUOUS:
        a, w = p[:n], p[n:]
        return np.where(np.all(X < w, axis=1), np.exp(X @ a), 0.0)
    if family == BOX_POWER:
        return np.sum(X * X, axis=1) ** p[0]
    raise ValueError


def gl_nodes(breaks, m):
    x, wt = np.polynomial.legendre.leggauss(m)
    xs, ws = [], []
    for lo, hi in zip(breaks[:-1], breaks[1:]):
        xs.append(lo + (hi - lo) * (x + 1) / 2)
        ws.append(wt * (hi - lo) / 2)
    return np.concatenate(xs), np.concatenate(ws)


def tensor_gl(family, n, p, panels=16, m=12, lo=None, hi=None):
    per_axis = []
    for j in range(n):
        a_j = 0.0 if lo is None else lo[j]
        b_j = 1.0 if hi is None else hi[j]
        br = list(np.linspace(a_j, b_j, panels + 1))
        if family in (C0, GAUSSIAN, PRODUCT_PEAK, DISCONTINUOUS):
            w = p[n + j]
            if a_j < w < b_j:
                br = sorted(set(br + [w]))
        per_axis.append(gl_nodes(np.array(br), m))
    grids = np.meshgrid(*[a[0] for a in per_axis], indexing="ij")
    wgrid = np.ones_like(grids[0])
    for j, g in enumerate(np.meshgrid(*[a[1] for a in per_axis], indexing="ij")):
        wgrid = wgrid * g
    X = np.stack([g.ravel() for g in grids], axis=1)
    return float(np.sum(wgrid.ravel() * f_numpy(family, n, p, X)))


@pytest.mark.parametrize("family", [PRODUCT_PEAK, GAUSSIAN, OSCILLATORY, CORNER_PEAK, C0, DISCONTINUOUS, BOX_POWER])
@pytest.mark.parametrize("n", [2, 3])
def test_closed_form_vs_gauss_legendre(family, n):
    p = draw_params(family, n, 9000 + 10 * family + n)
    if family == BOX_POWER:
        p = [float(round(p[0]))]      # integer exponent: the multinomial closed form
    panels, m = (16, 12) if n == 2 else (8, 10)
    ref = tensor_gl(family, n, p, panels, m)
    assert abs(cf.closed_form(family, n, p) - ref) <= 1e-10 * abs(ref)


@pytest.mark.parametrize("a", [0.5, 1.0, 2.0, 7.0])
def test_corner_peak_1d(a):
    # int_0^1 (1 + a x)^-2 dx = 1/(1 + a)
    assert abs(cf.closed_form(CORNER_PEAK, 1, [a]) - 1 / (1 + a)) < 1e-15


def test_golden_paper_integrands_are_reproduced():
    d = json.load(open(os.path.join(GOLDEN, "paper_integrands.json")))
    for c in d["cases"]:
        assert cf.closed_form(c["family"], c["dim"], c["params"]) == float(c["integral"])


def test_gaussian_closed_form_special_case():
    # with w = 1/2 each factor is sqrt(pi)/a * erf(a/2)
    a = 25.0
    v = cf.closed_form(GAUSSIAN, 1, [a, 0.5])
    assert abs(v - math.sqrt(math.pi) / a * math.erf(a / 2)) < 1e-16


@pytest.mark.parametrize("q", [0, 1, 2])
def test_box_power_small_exponents(q):
    # (sum x^2)^0 = 1; int sum x_j^2 = n/3; int (sum x_j^2)^2 = n/5 + n(n-1)/9
    n = 4
    ref = {0: 1.0, 1: n / 3, 2: n / 5 + n * (n - 1) / 9}[q]
    assert abs(cf.closed_form(BOX_POWER, n, [q]) - ref) < 1e-15 * ref
    assert cf.closed_form(BOX_POWER, n, [7.5]) is None


def test_discontinuous_jump_outside_the_cube():
    # w_j >= 1 on every axis: no jump inside, a plain product of exponentials
    a = [1.5, 2.5]
    v = cf.closed_form(DISCONTINUOUS, 2, a + [1.0, 3.0])
    assert abs(v - math.expm1(1.5) / 1.5 * math.expm1(2.5) / 2.5) < 1e-15 * v


@pytest.mark.parametrize("n,tau", [(2, 1e-10), (3, 1e-9)])
def test_oracle_box_power_half_integer_vs_quadrature(n, tau):
    """(sum x^2)^7.5 (paper f8's exponent) has no closed form; (r^2)^7.5 =
    r^15 is smooth enough that composite tensor Gauss-Legendre reaches 1e-13,
    which the oracle's converged estimate must match within its tolerance.
    (Its error estimate here is far below the rounding of the sum: after
    the first iteration nearly every null value sits under its noise
    floor.)"""
    ref = tensor_gl(BOX_POWER, n, [7.5], panels=16 if n == 2 else 8, m=12)
    o = capi.integrate(BOX_POWER, n, [7.5], tau, max_regions=1_000_000)
    assert o.status == 0
    assert abs(o.estimate - ref) <= tau * abs(ref)


def random_box(family, n, seed):
    """Bounds with negative and positive ends; the corner peak stays where
    1 + a.x > 0 (lower ends >= 0)."""
    rng = np.random.default_rng(seed)
    lo = rng.uniform(0.0, 0.5, n) if family == CORNER_PEAK else rng.uniform(-0.8, 0.6, n)
    hi = lo + rng.uniform(0.3, 1.4, n)
    return lo, hi


@pytest.mark.parametrize("family", [PRODUCT_PEAK, GAUSSIAN, OSCILLATORY, CORNER_PEAK, C0, DISCONTINUOUS, BOX_POWER])
@pytest.mark.parametrize("n", [2, 3])
def test_closed_form_box_vs_gauss_legendre(family, n):
    p = draw_params(family, n, 9100 + 10 * family + n)
    if family == BOX_POWER:
        p = [float(round(p[0]))]
    lo, hi = random_box(family, n, 77 + 10 * family + n)
    panels, m = (16, 12) if n == 2 else (8, 10)
    ref = tensor_gl(family, n, p, panels, m, lo, hi)
    assert abs(cf.closed_form_box(family, n, p, lo, hi) - ref) <= 1e-10 * abs(ref)


def test_closed_form_box_on_unit_cube_is_closed_form():
    for family in range(7):
        p = draw_params(family, 3, 4242 + family)
        if family == BOX_POWER:
            p = [6.0]
        a, b = cf.closed_form(family, 3, p), cf.closed_form_box(family, 3, p, [0.0] * 3, [1.0] * 3)
        assert abs(a - b) <= 1e-14 * abs(a)


@pytest.mark.parametrize("family", [PRODUCT_PEAK, GAUSSIAN, OSCILLATORY, C0, CORNER_PEAK])
def test_oracle_integrates_over_general_bounds(family):
    """Algorithm 2 over [a, b]: the Uniform-Split starts from the box, and the
    estimate lands within its error estimate of the box's closed form.  (The
    discontinuous family is left out: a box cut by the jump whose rule points
    all fall on the zero side reports V = E = 0, so its estimate can stop
    short with a vanishing error estimate -- 0.65 % off here, on any bounds.)"""
    n = 3
    p = draw_params(family, n, 9300 + family)
    lo, hi = random_box(family, n, 500 + family)
    o = capi.integrate(family, n, p, 1e-6, max_regions=2_000_000, relerr_filter=0 if family == OSCILLATORY else 1,
                       bounds=(lo, hi), want_regions=True)
    ex = cf.closed_form_box(family, n, p, lo, hi)
    assert o.status in (0, 3)
    if family == C0:
        # the null rules do not see the kink at w inside a box, so the
        # estimate is not a bound there (on the unit cube too); the requested
        # tolerance is still met
        assert abs(o.estimate - ex) <= 1e-6 * abs(ex), (o.estimate, ex, o.errorest)
    else:
        assert abs(o.estimate - ex) <= max(o.errorest, 1e-13 * abs(ex)), (o.estimate, ex, o.errorest)
    # the last iteration's regions and the finished ones tile [a, b]
    vol = np.prod(hi - lo)
    act = float(np.sum(np.prod(o.final_width, axis=1)))
    assert abs(act + o.finished_volume - vol) <= 1e-13 * vol
    assert np.all(o.final_lower >= lo) and np.all(o.final_lower + o.final_width <= hi * (1 + 1e-15))
