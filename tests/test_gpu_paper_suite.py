"""The paper's fixed-parameter test integrands f1..f8 (Sec. 4.1, mapped onto
the families in workloads.paper_integrands) as a regression suite: the GPU
loop against the oracle on each (statuses, iterations, region counts,
per-iteration trace, estimates within 1e-12), and the closed form (where one
exists) inside the reported error estimate exactly when it is inside the
oracle's.

The tolerances and pools are chosen so the oracle finishes each case in
seconds; several cases end in status 3 (the finished error alone exceeds the
tolerance) because the heuristic filter of Sec. 3.5.3 finishes boxes whose
errors add up past it, which is part of what is being checked."""
import pytest

from oracle import capi as oracle, closed_forms as cf
from paper_2104_06494_gb300.workloads import paper_integrands
from tests.conftest import has_gpu
from tests.gpu_util import compare_runs

pytestmark = pytest.mark.gpu

# name, epsrel, max_regions
SUITE = [
    ("f1_d8", 1e-3, 1_000_000),     # oscillatory, relative-error filter off: status 3
    ("f2_d6", 1e-2, 1_000_000),     # product peak c = 50: 11 iterations, 3.4e5 regions
    ("f3_d3", 1e-6, 1_000_000),     # corner peak: converged in one pass
    ("f3_d8", 1e-3, 1_000_000),
    ("f4_d5", 1e-3, 1_000_000),     # Gaussian a = 25: 1.05e6 regions over 12 iterations
    ("f5_d5", 1e-5, 1_000_000),     # C0
    ("f6_d6", 1e-3, 1_000_000),     # discontinuous: status 3 after 14 iterations
    ("f7_d8", 1e-6, 1_000_000),     # box power q = 11
    ("f8_d8", 1e-8, 1_000_000),     # box power q = 7.5 (no closed form)
]


@pytest.fixture(scope="module")
def pg():
    if not has_gpu():
        pytest.skip("no CUDA device")
    import paper_2104_06494_gb300 as m
    m.load()
    return m


@pytest.mark.parametrize("name,tau,max_regions", SUITE)
def test_paper_integrand_matches_oracle(pg, name, tau, max_regions):
    w = paper_integrands()[name]
    o = oracle.integrate(w.family, w.dim, w.params, tau, max_regions=max_regions, relerr_filter=w.relerr_filter)
    g = pg.pagani_integrate_ex(w.dim, w.family, w.params, tau, max_regions=max_regions,
                               relerr_filter=w.relerr_filter, trace=True)
    compare_runs(g, o)
    ex = cf.closed_form(w.family, w.dim, w.params)
    if ex is not None:
        assert (abs(g.estimate - ex) <= g.errorest) == (abs(o.estimate - ex) <= o.errorest)
