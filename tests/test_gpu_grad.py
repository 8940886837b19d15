"""GPU differentiation (the differentiation row of the build): the converged
leaf set kept by the integration equals the oracle's, the gradient kernel
matches the oracle's gradient on identical leaves, the torch.autograd
Function returns it, and on the d = 6 parametric Gaussian (theta = (a, w),
epsrel 1e-7) the gradient agrees with the closed-form erf gradient and with
central finite differences (h = 1e-5) of the frozen-leaf estimate and of the
full adaptive integration."""
import math

import numpy as np
import pytest

from oracle import capi as oracle, closed_forms as cf
from paper_2104_06494_gb300.workloads import config_workloads, draw_params
from tests.conftest import has_gpu
from tests.gpu_util import EPS, point_count

pytestmark = pytest.mark.gpu

RANGES = {0: [("n", 5.0, 10.0), ("n", 0.2, 0.8)], 1: [("n", 5.0, 15.0), ("n", 0.2, 0.8)],
          4: [("n", 1.0, 5.0), ("n", 0.2, 0.8)]}


@pytest.fixture(scope="module")
def pg():
    if not has_gpu():
        pytest.skip("no CUDA device")
    import paper_2104_06494_gb300 as m
    m.load()
    return m


def gpu_leaves_rows(pg, n):
    lower, level = pg.pagani_leaves(n)
    lo = lower.cpu().numpy().T
    wd = np.ldexp(1.0, -level.cpu().numpy().T.astype(np.int64))
    return lo, wd, lower, level


def sorted_rows(lo, wd):
    keys = np.concatenate([lo, wd], axis=1)
    return keys[np.lexsort(keys.T[::-1])]


def kappa(family, n, p):
    """Largest rounding sensitivity of f over the cube (as in value_condition)."""
    p = np.asarray(p)
    if family == 1:
        return float(np.sum(p[:n] ** 2 * np.maximum(p[n:], 1 - p[n:]) ** 2))
    if family == 4:
        return float(np.sum(p[:n] * np.maximum(p[n:], 1 - p[n:])))
    return 2.0 * n + 4


@pytest.mark.parametrize("family,n,tau", [(1, 3, 1e-7), (0, 2, 1e-6), (4, 3, 1e-4), (1, 5, 1e-5)])
def test_leaf_set_and_gradient_match_oracle(pg, family, n, tau):
    p = draw_params(family, n, 300 + family + n, RANGES[family])
    r = pg.pagani_integrate_ex(n, family, p, tau, max_regions=4_000_000, keep_leaves=1)
    o = oracle.integrate(family, n, p, tau, max_regions=4_000_000, want_leaves=True, parallel=True)
    assert r.status == o.status and r.n_regions == o.n_regions
    lo, wd, lower, level = gpu_leaves_rows(pg, n)
    assert r.n_leaves == len(lo) == len(o.leaves[0])
    assert np.array_equal(sorted_rows(lo, wd), sorted_rows(*o.leaves))
    v, g = pg.pagani_gradient(n, family, p, lower, level)
    vo, go, ab = oracle.gradient(family, n, p, lo, wd)
    tol = (point_count(n) + 4 * n + 32 + kappa(family, n, p)) * EPS
    assert abs(v - vo) <= 1e-12 * abs(vo) + tol * ab[0]
    assert abs(v - r.estimate) <= 1e-12 * abs(r.estimate) + tol * ab[0]
    for k in range(2 * n):
        assert abs(g[k] - go[k]) <= 1e-12 * abs(go[k]) + tol * ab[1 + k], (k, g[k], go[k])


def test_autograd_function(pg):
    import torch
    from paper_2104_06494_gb300.autograd import integral
    n = 3
    p = draw_params(1, n, 5, RANGES[1])
    theta = torch.tensor(p, dtype=torch.float64, requires_grad=True)
    I = integral(theta, n, 1, 1e-7)
    I.backward()
    r = pg.pagani_integrate_ex(n, 1, p, 1e-7, keep_leaves=1)
    _, _, lower, level = gpu_leaves_rows(pg, n)
    v, g = pg.pagani_gradient(n, 1, p, lower, level)
    assert float(I.detach()) == r.estimate
    assert np.allclose(theta.grad.numpy(), g, rtol=1e-13, atol=0)


def test_gradient_refuses_non_product_family(pg):
    import torch
    lower = torch.zeros((3, 1), dtype=torch.float64, device="cuda")
    level = torch.zeros((3, 1), dtype=torch.uint8, device="cuda")
    with pytest.raises(pg.PaganiError):
        pg.pagani_gradient(3, 3, [1.0, 1.0, 1.0], lower, level)


def test_differentiation_workload_d6(pg):
    """theta = (a_1..a_6, w_1..w_6), a ~ U[5,15], w ~ U[0.2,0.8], epsrel 1e-7."""
    w = config_workloads()["gaussian_d6_grad"]
    n, p = w.dim, np.array(w.params)
    r = pg.pagani_integrate_ex(n, w.family, p, w.epsrel, w.epsabs, w.max_regions, keep_leaves=1)
    assert r.n_leaves > 0
    _, _, lower, level = gpu_leaves_rows(pg, n)
    v, g = pg.pagani_gradient(n, w.family, p, lower, level)
    tot, gc = cf.gaussian_gradient(n, p)
    gc = np.array(gc)
    assert abs(r.estimate - tot) <= r.errorest
    # against the closed-form erf gradient, within the bound the integral's
    # error estimate implies: on a box the rule's error on a Gaussian factor
    # of width 1/a_j behaves like (a_j h)^10, so its derivative in a_j is
    # about 10 err / a_j, and in w_j (a shift by a fraction of the width
    # 1/a_j) about 10 a_j err; plus the rounding of the sums on the natural
    # scales |I| and a_j |I| of the two kinds of component
    a = p[:n]
    scale = np.concatenate([np.full(n, abs(tot)), a * abs(tot)])
    bound = np.concatenate([10 * r.errorest / a, 10 * r.errorest * a]) + 64 * EPS * scale
    assert np.all(np.abs(g - gc) <= bound), np.abs(g - gc) / bound
    # central differences h = 1e-5 of the estimate on the frozen leaf set
    h = 1e-5
    for k in range(2 * n):
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (pg.pagani_gradient(n, w.family, pp, lower, level)[0] -
              pg.pagani_gradient(n, w.family, pm, lower, level)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * abs(g[k]) + 64 * EPS * abs(tot) / h, (k, fd, g[k])
    # and of the full adaptive integration (each side adapts its own regions,
    # so the difference also carries both sides' integration errors / 2h)
    for k in (0, n):
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        rp = pg.pagani_integrate_ex(n, w.family, pp, w.epsrel, w.epsabs, w.max_regions)
        rm = pg.pagani_integrate_ex(n, w.family, pm, w.epsrel, w.epsabs, w.max_regions)
        fd = (rp.estimate - rm.estimate) / (2 * h)
        assert abs(fd - g[k]) <= (rp.errorest + rm.errorest) / (2 * h) + 1e-6 * abs(g[k]), (k, fd, g[k])


@pytest.mark.parametrize("family,n", [(1, 2), (0, 5), (4, 5), (1, 8)])
def test_gradient_on_deep_boxes_matches_oracle(pg, family, n):
    """Random dyadic boxes with levels up to 30 per axis: intervals of level
    11 or less take their factor values and chain-rule terms from the
    tables filled for the call, deeper ones compute them in place.  Both
    must give the oracle's point-by-point gradient on the same boxes."""
    import torch
    from paper_2104_06494_gb300.workloads import random_dyadic_regions
    m = 3000 if n < 8 else 400
    lo_l, wd_l = random_dyadic_regions(n, m, seed=900 + 10 * family + n, max_level=30)
    lo, wd = np.array(lo_l), np.array(wd_l)
    lv = np.rint(-np.log2(wd)).astype(np.uint8)
    assert lv.max() > 11 and lv.min() <= 11
    p = draw_params(family, n, 400 + family + n, RANGES[family])
    lower = torch.tensor(lo.T.copy(), dtype=torch.float64, device="cuda")
    level = torch.tensor(lv.T.copy(), dtype=torch.uint8, device="cuda")
    v, g = pg.pagani_gradient(n, family, p, lower, level)
    vo, go, ab = oracle.gradient(family, n, p, lo, wd)
    tol = (point_count(n) + 4 * n + 32 + kappa(family, n, p)) * EPS
    assert abs(v - vo) <= 1e-12 * abs(vo) + tol * ab[0]
    for k in range(2 * n):
        assert abs(g[k] - go[k]) <= 1e-12 * abs(go[k]) + tol * ab[1 + k], (k, g[k], go[k])
