"""GPU parity of the whole PAGANI loop (Algorithm 2 with Algorithm 3) through
the C ABI against the oracle on the same seeded inputs: equal iteration
counts, region counts and statuses, estimates within 1e-12 relative, and a
per-iteration trace diff; plus graph vs host-driven loop, bitwise
repeatability, the failure statuses and closed-form containment."""
import numpy as np
import pytest

from oracle import capi as oracle, closed_forms as cf
from paper_2104_06494_gb300.workloads import config_workloads, draw_params
from tests.conftest import has_gpu
from tests.gpu_util import close, compare_runs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg():
    if not has_gpu():
        pytest.skip("no CUDA device")
    import paper_2104_06494_gb300 as m
    m.load()
    return m


CASES = [
    (0, 2, 1e-6, 1), (0, 3, 1e-3, 1), (0, 4, 1e-6, 1),
    (1, 2, 1e-7, 1), (1, 3, 1e-5, 1), (1, 5, 1e-4, 1),
    (2, 2, 1e-8, 0), (2, 3, 1e-7, 0), (2, 6, 1e-6, 0),
    (3, 3, 1e-7, 1), (3, 5, 1e-6, 1), (3, 8, 1e-3, 1),
    (4, 2, 1e-5, 1), (4, 3, 1e-4, 1), (4, 8, 1e-3, 1),
    # the box power at tolerances down to 1e-11: below about 5e-13 (n = 3) the
    # tolerance sits under the null values' own noise floor, 64 N(n) u of
    # their sums, and rounding decides the classification on either side
    (5, 4, 1e-3, 1), (6, 3, 1e-11, 1), (6, 5, 1e-10, 1), (6, 8, 1e-7, 1),
]


@pytest.mark.parametrize("family,n,tau,relerr", CASES)
def test_loop_matches_oracle(pg, family, n, tau, relerr):
    # C0 in 8-D runs out of a 10^6 pool after 15 iterations (1.5e6 regions
    # evaluated): memory-exhaustion parity at a size the oracle takes seconds on
    pool = 1_000_000 if (family, n) == (4, 8) else 4_000_000
    params = draw_params(family, n, 700 + 13 * family + n)
    o = oracle.integrate(family, n, params, tau, max_regions=pool, relerr_filter=relerr, parallel=True)
    g = pg.pagani_integrate_ex(n, family, params, tau, max_regions=pool, relerr_filter=relerr, trace=True)
    compare_runs(g, o, value_scale=1.0 if family == 2 else 0.0)


def _box(family, n, seed, params=None):
    """A random box with negative and positive ends; the corner peak's stays
    where 1 + a.x > 0, and with params given the Gaussian's holds its peak w
    (a box far from a narrow peak leaves the first rule points in its tail,
    where the error estimate is blind: at d = 8 such a box gave 1e-83 for
    an integral of 5e-74, with an error estimate of 2e-85, on both sides)."""
    rng = np.random.default_rng(seed)
    if family == 1 and params is not None:
        w = np.asarray(params[n:2 * n])
        return w - rng.uniform(0.3, 0.7, n), w + rng.uniform(0.3, 0.7, n)
    lo = rng.uniform(0.0, 0.5, n) if family == 3 else rng.uniform(-0.8, 0.6, n)
    return lo, lo + rng.uniform(0.3, 1.4, n)


@pytest.mark.parametrize("family,n,tau", [(0, 3, 1e-6), (1, 4, 1e-5), (2, 3, 1e-6), (3, 3, 1e-7), (4, 3, 1e-4),
                                          (5, 3, 1e-3), (6, 3, 1e-9), (1, 6, 1e-4), (1, 8, 1e-2)])
def test_general_bounds_match_oracle(pg, family, n, tau):
    """Algorithm 2 over a box [a, b] with negative and positive ends: the GPU
    maps unit-cube rule points onto the box, the oracle splits the box
    itself; equal region sets and traces, estimates to 1e-12, the volume
    of the box tiled, and the box's closed form inside the error estimate
    (except for the C0 kink and the discontinuous jump, where the null rules
    are not a bound)."""
    params = draw_params(family, n, 1700 + 10 * family + n)
    lo, hi = _box(family, n, 41 + 10 * family + n, params)
    relerr = 0 if family == 2 else 1
    o = oracle.integrate(family, n, params, tau, max_regions=2_000_000, relerr_filter=relerr, bounds=(lo, hi), parallel=True)
    g = pg.pagani_integrate_ex(n, family, params, tau, max_regions=2_000_000, relerr_filter=relerr,
                               bounds=(lo, hi), trace=True)
    compare_runs(g, o)
    vol = float(np.prod(hi - lo))
    assert abs(g.finished_volume + g.active_volume - vol) <= 1e-13 * vol
    assert abs(g.finished_volume - o.finished_volume) <= 1e-13 * vol
    ex = cf.closed_form_box(family, n, params, lo, hi)
    if ex is not None and family not in (4, 5):
        assert abs(g.estimate - ex) <= max(g.errorest, 1e-13 * abs(ex))


def test_unit_bounds_are_the_unit_cube_bitwise(pg):
    """The map lo + len x with lo = 0, len = 1 is exact, so integrating over
    [0, 1]^n through the bounds entry gives the unit-cube run bit for bit."""
    for family, n in ((1, 5), (2, 4), (6, 3)):
        params = draw_params(family, n, 88 + family)
        a = pg.pagani_integrate_ex(n, family, params, 1e-6, relerr_filter=0 if family == 2 else 1, trace=True)
        b = pg.pagani_integrate_ex(n, family, params, 1e-6, relerr_filter=0 if family == 2 else 1, trace=True,
                                   bounds=(np.zeros(n), np.ones(n)))
        assert (a.estimate, a.errorest, a.status, a.n_regions) == (b.estimate, b.errorest, b.status, b.n_regions)
        assert a.trace.tobytes() == b.trace.tobytes()


def test_bounds_scale_the_measure(pg):
    """Integrating f(x) over [a, b] equals vol * the integral of f(a + L t)
    over the unit cube: for the Gaussian, the latter is itself a Gaussian with
    a' = a L and w' = (w - a)/L.  The two runs see the same values up to
    rounding, but the bounded run breaks split-axis ties by widths on the
    box, so their region sets may differ; the estimates agree within the
    two error estimates."""
    n = 4
    p = np.array(draw_params(1, n, 5151))
    lo, hi = _box(1, n, 5, p)
    L = hi - lo
    a, w = p[:n], p[n:]
    g = pg.pagani_integrate_ex(n, 1, p, 1e-7, bounds=(lo, hi))
    u = pg.pagani_integrate_ex(n, 1, np.concatenate([a * L, (w - lo) / L]), 1e-7)
    vol = float(np.prod(L))
    assert g.status == u.status
    assert abs(g.estimate - vol * u.estimate) <= g.errorest + vol * u.errorest


def test_bounds_argument_errors(pg):
    with pytest.raises(pg.PaganiError, match="-8"):
        pg.pagani_integrate_ex(3, 1, draw_params(1, 3, 1), 1e-3, bounds=([0, 0, 0], [1, 0, 1]))
    with pytest.raises(pg.PaganiError, match="-8"):
        pg.pagani_integrate_ex(3, 1, draw_params(1, 3, 1), 1e-3, bounds=([0, 0, 0], [1, np.inf, 1]))


GM7_CASES = [(0, 3, 1e-6), (1, 4, 1e-5), (1, 6, 1e-4), (2, 3, 1e-7), (3, 5, 1e-6), (4, 3, 1e-4), (5, 3, 1e-3),
             (6, 5, 1e-9)]


@pytest.mark.parametrize("family,n,tau", GM7_CASES)
def test_gm7_loop_matches_oracle(pg, family, n, tau):
    """The whole loop with the Genz-Malik degree-7 rule (error |R7 - R5|):
    equal region sets, traces and estimates, and the closed form inside the
    error estimate where the oracle's is (all but the discontinuous case)."""
    params = draw_params(family, n, 800 + 13 * family + n)
    relerr = 0 if family == 2 else 1
    o = oracle.integrate(family, n, params, tau, max_regions=4_000_000, relerr_filter=relerr, degree=7, parallel=True)
    g = pg.pagani_integrate_ex(n, family, params, tau, max_regions=4_000_000, relerr_filter=relerr, trace=True,
                               rule_degree=7)
    compare_runs(g, o)
    ex = cf.closed_form(family, n, params)
    if ex is not None and family != 5:
        assert abs(g.estimate - ex) <= g.errorest


def test_gm7_uses_fewer_points_per_region(pg):
    """Same integral, both rules: the degree-7 run evaluates
    2^n + 2n^2 + 2n + 1 points per region (401 at n = 8, against 1105) and
    both estimates hold the closed form within their error estimates (the
    degree-7 run, whose error is the plain |R7 - R5|, runs out of the 2^24
    pool before its estimate reaches 1e-3)."""
    n = 8
    params = draw_params(1, n, 8080)
    ex = cf.closed_form(1, n, params)
    r9 = pg.pagani_integrate_ex(n, 1, params, 1e-3, max_regions=1 << 24)
    r7 = pg.pagani_integrate_ex(n, 1, params, 1e-3, max_regions=1 << 24, rule_degree=7)
    for r in (r9, r7):
        assert r.status in (0, 2) and abs(r.estimate - ex) <= r.errorest


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_filter_modes_match_oracle(pg, mode):
    """The filtering ablation (Sec. 4.2): Threshold-Classify off (0), on with
    both triggers of Sec. 3.5.2 (1), with the memory trigger only (2) or the
    unchanged-digits trigger only (3), on the paper's f4 at d = 5 with a
    10^6-region pool: modes 1 and 2 converge, 0 and 3 run out of memory at
    iteration 10, on both sides alike."""
    from paper_2104_06494_gb300.workloads import paper_integrands
    w = paper_integrands()["f4_d5"]
    o = oracle.integrate(w.family, w.dim, w.params, 1e-4, max_regions=1_000_000, heuristic_filter=mode, parallel=True)
    g = pg.pagani_integrate_ex(w.dim, w.family, w.params, 1e-4, max_regions=1_000_000, heuristic_filter=mode,
                               trace=True)
    compare_runs(g, o)
    assert g.status == (0 if mode in (1, 2) else 2)


def test_filtering_ablation_f4_d8(pg):
    """The paper's ablation case: 8-D f4 at three digits.  With the heuristic
    filter the run converges inside a 2^27-region pool; without it the
    active set outgrows the pool (memory exhausted, status 2) before the
    error estimate reaches 1e-3."""
    from paper_2104_06494_gb300.workloads import paper_integrands
    w = paper_integrands()["f4_d8"]
    ex = cf.closed_form(w.family, w.dim, w.params)
    on = pg.pagani_integrate_ex(w.dim, w.family, w.params, 1e-3, max_regions=1 << 27, heuristic_filter=1)
    off = pg.pagani_integrate_ex(w.dim, w.family, w.params, 1e-3, max_regions=1 << 27, heuristic_filter=0)
    assert on.status == 0 and abs(on.estimate - ex) <= on.errorest
    assert off.status == 2 and off.errorest > 1e-3 * abs(off.estimate)


@pytest.mark.parametrize("n,tau", [(2, 1e-4), (3, 1e-3)])
def test_discontinuous_without_heuristic_filter(pg, n, tau):
    """The discontinuous family with the heuristic filter off: millions of
    regions, the pool grown and compacted over 20 or more iterations, equal
    on both sides.  At d = 2 the loop converges with the closed form inside
    the estimate; at d = 3 the boxes cut by the jump keep their large
    errors until the 4e6-region pool is exhausted (status 2), and the
    estimate still covers the true error."""
    family = 5
    params = draw_params(family, n, 700 + 13 * family + n)
    o = oracle.integrate(family, n, params, tau, max_regions=4_000_000, heuristic_filter=0, parallel=True)
    g = pg.pagani_integrate_ex(n, family, params, tau, max_regions=4_000_000, heuristic_filter=0, trace=True)
    assert o.status == (0 if n == 2 else 2)
    compare_runs(g, o)
    ex = cf.closed_form(family, n, params)
    assert abs(g.estimate - ex) <= g.errorest


def test_config_product_peak_d3_full_size(pg):
    """The d=3 product-peak workload at its full size (epsrel 1e-3, 1e5 regions)."""
    w = config_workloads()["product_peak_d3"]
    o = oracle.integrate(w.family, w.dim, w.params, w.epsrel, w.epsabs, w.max_regions, parallel=True)
    g = pg.pagani_integrate_ex(w.dim, w.family, w.params, w.epsrel, w.epsabs, w.max_regions, trace=True)
    compare_runs(g, o)
    ex = cf.closed_form(w.family, w.dim, w.params)
    assert abs(g.estimate - ex) <= g.errorest and g.status == 0


@pytest.mark.parametrize("n", [2, 5, 8])
def test_zero_and_constant_integrands(pg, n):
    """Degenerate integrands: f = 0 converges in one pass with estimate and
    error exactly 0; f = 1 returns the volume, to the rounding of the double
    weights' sum (the oracle, summing exact-rounded weights per orbit, gets 1
    exactly; the kernel's order is 1 ulp off at n = 8), with an error
    estimate at the rounding level of the rule sums, 16 u sum_g |w_g| cnt_g,
    as the oracle's."""
    g = pg.pagani_integrate_ex(n, 5, [1.0] * n + [0.0] * n, 1e-6)
    assert (g.status, g.iterations, g.estimate, g.errorest) == (0, 1, 0.0, 0.0)
    g = pg.pagani_integrate_ex(n, 6, [0.0], 1e-12)
    o = oracle.integrate(6, n, [0.0], 1e-12, parallel=True)
    assert (g.status, g.iterations) == (0, 1)
    assert abs(g.estimate - 1.0) <= 4 * 2.0 ** -53
    assert 0.0 < g.errorest and abs(g.errorest - o.errorest) <= 1e-12 * o.errorest


@pytest.mark.parametrize("init_div", [2, 8])
def test_non_default_uniform_split_matches_oracle(pg, init_div):
    params = [10.0, 12.0, 14.0, 0.3, 0.5, 0.7]
    o = oracle.integrate(1, 3, params, 1e-6, init_div=init_div, parallel=True)
    g = pg.pagani_integrate_ex(3, 1, params, 1e-6, init_div=init_div, trace=True)
    compare_runs(g, o)


def test_graph_and_host_loop_identical(pg):
    params = draw_params(1, 4, 42)
    a = pg.pagani_integrate_ex(4, 1, params, 1e-6, use_graph=1, trace=True)
    b = pg.pagani_integrate_ex(4, 1, params, 1e-6, use_graph=0, trace=True)
    assert (a.estimate, a.errorest, a.status, a.iterations, a.n_regions) == \
           (b.estimate, b.errorest, b.status, b.iterations, b.n_regions)
    assert a.trace.tobytes() == b.trace.tobytes()


def test_bitwise_repeatable(pg):
    params = draw_params(4, 5, 43)
    r = [pg.pagani_integrate_ex(5, 4, params, 1e-4, trace=True) for _ in range(3)]
    for x in r[1:]:
        assert (x.estimate, x.errorest, x.n_regions) == (r[0].estimate, r[0].errorest, r[0].n_regions)


def test_memory_exhausted_matches_oracle(pg):
    params = draw_params(1, 3, 3)
    o = oracle.integrate(1, 3, params, 1e-12, max_regions=6000, heuristic_filter=0, parallel=True)
    g = pg.pagani_integrate_ex(3, 1, params, 1e-12, max_regions=6000, heuristic_filter=0, trace=True)
    assert o.status == 2
    compare_runs(g, o)


def test_it_max_and_capacity(pg):
    params = draw_params(1, 3, 3)
    g = pg.pagani_integrate_ex(3, 1, params, 1e-12, it_max=1)
    assert g.status == 1 and g.iterations == 1 and g.n_regions == 4096
    with pytest.raises(pg.PaganiError):
        pg.pagani_integrate(3, 1, params, 1e-3, max_regions=100)


def test_nonfinite_integrand(pg):
    g = pg.pagani_integrate_ex(2, 3, [-2.0, 0.5], 1e-3, raise_on_error=False)
    assert g.status == -6


@pytest.mark.parametrize("name", ["product_peak_d3", "oscillatory_d6", "corner_peak_d8"])
def test_configs_within_errorest_of_closed_form(pg, name):
    w = config_workloads()[name]
    g = pg.pagani_integrate_ex(w.dim, w.family, w.params, w.epsrel, w.epsabs, w.max_regions,
                               relerr_filter=w.relerr_filter)
    ex = cf.closed_form(w.family, w.dim, w.params)
    assert g.status == 0
    assert abs(g.estimate - ex) <= g.errorest


def test_bench_workload_gaussian_d5_full_size(pg):
    """The bench's 5-D Gaussian at its full size (epsrel 1e-7, 1.35e6
    regions over 18 iterations), in the launch configuration bench.py times
    (graph loop, library workspace): the same region-set evolution as the
    oracle, the estimate within 1e-12, converged with the closed form
    inside the estimate."""
    w = config_workloads()["gaussian_d5"]
    o = oracle.integrate(w.family, w.dim, w.params, w.epsrel, w.epsabs, w.max_regions, parallel=True)
    g = pg.pagani_integrate_ex(w.dim, w.family, w.params, w.epsrel, w.epsabs, w.max_regions, trace=True)
    compare_runs(g, o)
    ex = cf.closed_form(w.family, w.dim, w.params)
    assert abs(g.estimate - ex) <= g.errorest


def test_tens_of_millions_of_regions_per_iteration(pg):
    """A 3-D C0 integral (kinks at 0.31, 0.47, 0.73) at epsrel 1e-10 with
    the heuristic filter off and a pool of 2^25 regions: the active set
    grows to 2.5e7 regions and the pool runs out at iteration 23 (status 2),
    with 7.0e7 region evaluations in all.  At that size the count kernel
    gives each block more than one group of 8 tiles (its prefetched bytes
    cross groups), and the split forms the finished sums of millions of
    regions a launch.  Region-set evolution, trace and estimates as the
    oracle's."""
    params = [3.0, 4.0, 5.0, 0.31, 0.47, 0.73]
    o = oracle.integrate(4, 3, params, 1e-10, 1e-30, 1 << 25, heuristic_filter=0, it_max=40, parallel=True)
    g = pg.pagani_integrate_ex(3, 4, params, 1e-10, 1e-30, 1 << 25, heuristic_filter=0, it_max=40, trace=True)
    assert o.status == 2 and int(o.trace["s"].max()) > 2 * 10 ** 7
    compare_runs(g, o)
    ex = cf.closed_form(4, 3, params)
    assert abs(g.estimate - ex) <= g.errorest


def test_config_corner_peak_d8_loop_parity(pg):
    """The 8-D corner peak at epsrel 1e-3 (30 iterations, 6.7e5 regions of
    1105 points, threshold searches on the way): the same region-set
    evolution as the oracle.  At its full tolerance, 1e-6, the run takes
    1.7e8 region evaluations, beyond the oracle; it is checked by its
    properties below."""
    w = config_workloads()["corner_peak_d8"]
    o = oracle.integrate(w.family, w.dim, w.params, 1e-3, w.epsabs, w.max_regions, parallel=True)
    g = pg.pagani_integrate_ex(w.dim, w.family, w.params, 1e-3, w.epsabs, w.max_regions, trace=True)
    compare_runs(g, o)


@pytest.mark.parametrize("name", ["corner_peak_d8", "c0_d8"])
def test_config_d8_full_size_properties(pg, name):
    """The 8-D corner peak and C0 workloads at full size (epsrel 1e-6, pool
    capped at 4e8 regions), beyond the oracle; properties that hold at any
    size: the estimate within its error of the closed form (and within
    epsrel when converged), exact bookkeeping of the dyadic volume,
    s_{it+1} = 2 (survivors of it), and the finished error never above the
    tolerance."""
    w = config_workloads()[name]
    g = pg.pagani_integrate_ex(w.dim, w.family, w.params, w.epsrel, w.epsabs, w.max_regions, trace=True)
    ex = cf.closed_form(w.family, w.dim, w.params)
    assert g.status in ((0,) if name == "corner_peak_d8" else (0, 2))
    assert abs(g.estimate - ex) <= g.errorest
    if g.status == 0:
        assert abs(g.estimate - ex) <= w.epsrel * abs(ex)
    assert abs(g.finished_volume + g.active_volume - 1.0) <= 1e-13
    tr = g.trace
    for a, b in zip(tr[:-1], tr[1:]):
        assert b["s"] == 2 * a["n_survivors"]
    assert g.n_regions == int(tr["s"].sum())
    vf_old = 0.0
    for t in tr:
        assert t["ef"] <= w.epsrel * abs(t["v"] + vf_old) * (1 + 1e-3)
        vf_old = t["vf"]


def test_volume_bookkeeping_matches_oracle(pg):
    params = draw_params(1, 3, 61)
    o = oracle.integrate(1, 3, params, 1e-7, max_regions=2_000_000, want_regions=True, parallel=True)
    g = pg.pagani_integrate_ex(3, 1, params, 1e-7, max_regions=2_000_000)
    act = float(np.sum(np.prod(o.final_width, axis=1)))
    assert abs(g.finished_volume - o.finished_volume) <= 1e-15
    assert abs(g.active_volume - act) <= 1e-15
    assert abs(g.finished_volume + g.active_volume - 1.0) <= 1e-14
