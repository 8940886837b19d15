"""Pins of the oracle's differentiation: the closed-form gradient of the
Gaussian family against central differences of its closed form, the oracle's
rule gradient against central differences of its own rule sum on a frozen
box set (product peak, Gaussian, C0), and the leaf-set invariants."""
import numpy as np
import pytest

from oracle import capi, closed_forms as cf
from paper_2104_06494_gb300.workloads import draw_params, random_dyadic_regions

GRAD_FAMS = [0, 1, 4]
RANGES = {0: [("n", 5.0, 10.0), ("n", 0.2, 0.8)], 1: [("n", 5.0, 15.0), ("n", 0.2, 0.8)],
          4: [("n", 1.0, 5.0), ("n", 0.2, 0.8)]}


@pytest.mark.parametrize("n", [2, 3, 6])
def test_closed_form_gradient_vs_central_differences(n):
    p = np.array(draw_params(1, n, 70 + n, RANGES[1]))
    tot, g = cf.gaussian_gradient(n, p)
    assert abs(tot - cf.closed_form(1, n, p)) <= 1e-15 * abs(tot)
    for k in range(2 * n):
        h = 1e-6 * max(1.0, abs(p[k]))
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (cf.closed_form(1, n, pp) - cf.closed_form(1, n, pm)) / (2 * h)
        # truncation ~h^2, rounding of the difference 8 u |I| / h
        assert abs(fd - g[k]) <= 1e-6 * abs(g[k]) + 8 * 2.0 ** -53 * abs(tot) / h, (k, fd, g[k])


@pytest.mark.parametrize("family", GRAD_FAMS)
@pytest.mark.parametrize("n", [2, 4])
def test_rule_gradient_vs_central_differences_frozen_boxes(family, n):
    p = np.array(draw_params(family, n, 80 + family + n, RANGES[family]))
    lo, wd = random_dyadic_regions(n, 40, 3 + n, max_level=5)
    lo, wd = np.array(lo), np.array(wd)
    v, g, ab = capi.gradient(family, n, p, lo, wd)
    V, _, _ = capi.evaluate(family, n, p, lo, wd)
    assert abs(v - V.sum()) <= 1e-13 * ab[0]
    for k in range(2 * n):
        h = 1e-5 * max(1.0, abs(p[k]))
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (capi.gradient(family, n, pp, lo, wd)[0] - capi.gradient(family, n, pm, lo, wd)[0]) / (2 * h)
        # C0 is not differentiable where a rule point sits on the kink; its
        # points avoid w for these draws
        assert abs(fd - g[k]) <= 1e-6 * ab[1 + k] + 1e-9 * ab[0], (k, fd, g[k])


@pytest.mark.parametrize("family,n,tau", [(1, 3, 1e-7), (0, 2, 1e-6), (4, 3, 1e-4)])
def test_leaf_set_invariants(family, n, tau):
    p = draw_params(family, n, 90 + family, RANGES[family])
    r = capi.integrate(family, n, p, tau, max_regions=2_000_000, want_leaves=True)
    lo, wd = r.leaves
    assert abs(np.sum(np.prod(wd, axis=1)) - 1.0) <= 1e-14      # the leaves tile the cube
    v, g, ab = capi.gradient(family, n, p, lo, wd)
    assert abs(v - r.estimate) <= 1e-14 * ab[0]                   # and carry the estimate
    assert len(lo) == r.n_regions - int(np.sum(r.trace["n_survivors"][:-1]))


def test_gaussian_gradient_close_to_closed_form():
    n = 3
    p = draw_params(1, n, 5, RANGES[1])
    r = capi.integrate(1, n, p, 1e-8, max_regions=2_000_000, want_leaves=True)
    lo, wd = r.leaves
    _, g, _ = capi.gradient(1, n, p, lo, wd)
    _, gc = cf.gaussian_gradient(n, p)
    rel = np.abs(np.array(g) - np.array(gc)) / np.abs(gc)
    assert np.all(rel < 1e-4), rel
