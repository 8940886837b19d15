"""Pins of the oracle's error estimate (Sec. 3.2: the null-rule error and the
two-level refinement) against values that do not come from the estimate's
own formula: exact errors of polynomials, closed-form integrals of the
integrand families, and the error the method actually makes.

The estimate must bound the error (a converged result within its error
estimate of the closed form, Sec. 4.2 "Accuracy"), and must not overstate
it by orders of magnitude on a smooth integrand (Sec. 3.2 calls the
two-level estimate less susceptible to overestimation; an estimate inflated
a million times stops the loop from converging at all).

One blind spot of every fixed-point cubature error estimate is pinned as
such: a kink or jump inside the outer margin of a box, outside the span of
the rule's points, is seen by no null rule and by no parent-child
comparison."""
import multiprocessing as mp
from fractions import Fraction

import numpy as np
import pytest

from oracle import capi, closed_forms as cf, rule
from paper_2104_06494_gb300.workloads import (batch_workloads, config_workloads, draw_params,
                                              PRODUCT_PEAK, GAUSSIAN, OSCILLATORY, CORNER_PEAK, C0,
                                              SplitMix64)

FAMS = [PRODUCT_PEAK, GAUSSIAN, OSCILLATORY, CORNER_PEAK, C0]
MONOMIAL = 100  # oracle test family: prod_j x_j^(p_j)


def test_error_covers_the_exact_error_of_degree_10_to_14_polynomials():
    """The degree-9 rule's error on a polynomial of degree 10, 12 or 14 is
    known exactly (rational box integrals).  On dyadic boxes from width 1
    down to 1/32 (the asymptotic regime the ratio test reads) the region
    error must cover it.  A formula that dropped the safety factor, or that
    shrank the asymptotic branch as r^3, fails here on some boxes."""
    rng = SplitMix64(7)
    checked = 0
    for n in (2, 3, 5, 8):
        for _ in range(60):
            deg = 10 + 2 * int(rng.uniform(0, 3))
            p = [0] * n
            for _ in range(deg):
                p[int(rng.uniform(0, n))] += 1
            h = 2.0 ** -int(rng.uniform(0, 6))
            lo = [int(rng.uniform(0, 1 / h)) * h for _ in range(n)]
            V, E, K = capi.evaluate(MONOMIAL, n, [float(x) for x in p], [lo], [[h] * n])
            exact = Fraction(1)
            for j in range(n):
                a = Fraction(lo[j])
                b = a + Fraction(h)
                exact *= (b ** (p[j] + 1) - a ** (p[j] + 1)) / (p[j] + 1)
            err = abs(Fraction(V[0]) - exact)
            assert Fraction(E[0]) >= err, (n, p, h, lo, float(err), E[0])
            checked += err > 0
    assert checked > 200


def _run(args):
    family, n, params, tau, pool, relerr, parallel = args
    r = capi.integrate(family, n, params, tau, 1e-20, pool, relerr_filter=relerr, parallel=parallel)
    return r.status, r.estimate, r.errorest, cf.closed_form(family, n, params)


def _contained(status, est, err, exact, tau):
    """Within the error estimate; a converged result is also within tau."""
    ok = abs(est - exact) <= err
    if status == 0:
        ok = ok and abs(est - exact) <= max(err, tau * abs(exact))
    return ok


@pytest.mark.parametrize("n", [5, 6, 7, 8])
def test_estimates_within_errorest_in_five_to_eight_dimensions(n):
    """Every family on seeded parameters at tau 1e-4, 1e-6 and 1e-8, with a
    pool the oracle finishes in seconds: converged results carry their true
    error within the error estimate (and so within tau), and results that
    ran out of regions (status 2) still cover their error."""
    pool = {5: 1 << 16, 6: 1 << 15, 7: 1 << 14, 8: 1 << 13}[n]
    jobs = []
    for fam in FAMS:
        for k, tau in enumerate((1e-4, 1e-6, 1e-8)):
            p = draw_params(fam, n, 9100 + 31 * fam + 7 * n + k)
            jobs.append((fam, n, p, tau, pool, 0 if fam == OSCILLATORY else 1, True))
    for (fam, _, p, tau, *_), (st, est, err, exact) in zip(jobs, map(_run, jobs)):
        assert st in (0, 2), (fam, tau, st)
        assert _contained(st, est, err, exact, tau), (fam, n, tau, st, est - exact, err)


def test_batch_mix_sample_within_errorest():
    """A seeded sample of the batched workload (dimension 3..6, five
    families, tau in {1e-4, 1e-6, 1e-8}, 16384 regions per integral): no
    result outside its error estimate of the closed form, and no converged
    result further than tau from it."""
    items = [w for w in batch_workloads() if w.dim <= 6][::16]
    jobs = [(w.family, w.dim, w.params, w.epsrel, 16384, w.relerr_filter, False) for w in items]
    with mp.get_context("spawn").Pool(min(8, mp.cpu_count())) as pool:
        res = pool.map(_run, jobs, chunksize=2)
    bad = [(w.name, st, est - exact, err) for w, (st, est, err, exact) in zip(items, res)
           if not _contained(st, est, err, exact, w.epsrel)]
    assert len(items) > 150
    assert not bad, bad
    assert sum(st == 0 for st, *_ in res) > len(res) // 2


def test_error_estimate_is_not_orders_of_magnitude_pessimistic():
    """The 5-D Gaussian at tau 1e-7 (Gaussian peaks of width 1/5 to 1/15):
    the loop converges, the error estimate covers the true error and
    overstates it by less than 10^3; per iteration, the single-level region
    errors overstate the regions' summed absolute errors by less than 10^4.
    (A region error that fell back on the degree-1 null value wherever N_1
    >= N_2 overstated the converged error by 10^6 and kept the loop from
    converging.)"""
    w = config_workloads()["gaussian_d5"]
    exact = cf.closed_form(w.family, w.dim, w.params)
    r = capi.integrate(w.family, w.dim, w.params, w.epsrel, w.epsabs, w.max_regions, parallel=True)
    assert r.status == 0
    true_err = abs(r.estimate - exact)
    assert true_err <= r.errorest <= 1e3 * true_err
    r8 = capi.integrate(w.family, w.dim, w.params, w.epsrel, w.epsabs, w.max_regions, it_max=8,
                        want_regions=True, parallel=True)
    V, E, K = capi.evaluate(w.family, w.dim, w.params, r8.final_lower, r8.final_width)
    I = np.array([cf.closed_form_box(w.family, w.dim, w.params, lo, lo + wd)
                  for lo, wd in zip(r8.final_lower, r8.final_width)])
    assert np.sum(E) >= np.sum(np.abs(V - I))
    assert np.sum(E) <= 1e4 * np.sum(np.abs(V - I))


def test_kink_in_the_outer_margin_is_invisible():
    """C0 in 2-D at tau 1e-9 with these parameters: the kink line x_0 = w_0
    lies at 99.91 % of the width of a column of boxes [1/32, 3/64] along axis
    0, outside the span of the rule's points (the outermost radius is
    sqrt(l1) = 0.956 of the half-width).  Every rule point of those boxes
    sees a smooth exponential, so no null value and no parent-child
    comparison registers the sliver, and the converged result misses the
    closed form by more than its error estimate.  Pinned as a limitation:
    the whole shortfall sits in leaves whose kink lies outside their rule
    points' span, and every other leaf set is covered by its errors."""
    n = 2
    p = draw_params(C0, n, 100 + 7 * C0 + n)
    exact = cf.closed_form(C0, n, p)
    r = capi.integrate(C0, n, p, 1e-9, max_regions=2_000_000, want_leaves=True)
    assert r.status == 0 and abs(r.estimate - exact) > r.errorest
    lo, wd = r.leaves
    V, E, K = capi.evaluate(C0, n, p, lo, wd)
    I = np.array([cf.closed_form_box(C0, n, p, a, a + b) for a, b in zip(lo, wd)])
    reach = float(np.sqrt(float(rule.L1)))  # outermost rule radius per axis
    w = np.array(p[n:2 * n])
    rel = (w[None, :] - lo) / wd                      # kink position within the box, per axis
    inside = (rel > 0) & (rel < 1)
    seen = inside & (np.abs(rel - 0.5) < 0.5 * reach)
    blind = np.any(inside & ~seen, axis=1)
    assert np.sum(np.abs(V[~blind] - I[~blind])) <= np.sum(E[~blind])
    assert np.sum(V[blind] - I[blind]) > np.sum(E[blind])
    # the shortfall of the whole result is the blind leaves' error
    assert abs((r.estimate - exact) - np.sum(V[blind] - I[blind])) <= 1e-2 * abs(r.estimate - exact)
