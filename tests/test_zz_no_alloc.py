"""The allocation-free entry point, pagani_integrate_noalloc, for callers that
cannot allocate device memory (an application whose own allocator owns the
device, service loops that must never allocate).  It must give the same results as the
workspace path, pagani_integrate_ex, within the loop-parity tolerance of the
other GPU tests, on two calls in a row that share its static scratch array,
and it must refuse problems larger than that array with a clear error.

The file name sorts last so a run that stops at the first failure has already
run every other test."""
import pytest

from paper_2104_06494_gb300.workloads import config_workloads, draw_params
from tests.conftest import has_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg():
    if not has_gpu():
        pytest.skip("no CUDA device")
    import paper_2104_06494_gb300 as m
    m.load()
    return m


def same_result(a, b):
    assert a.status == b.status, (a.status, b.status)
    assert a.iterations == b.iterations and a.n_regions == b.n_regions and a.n_active_last == b.n_active_last
    assert abs(a.estimate - b.estimate) <= 1e-12 * abs(b.estimate) + 1e-300, (a.estimate, b.estimate)
    assert abs(a.errorest - b.errorest) <= 1e-6 * abs(b.errorest) + 1e-12 * abs(b.estimate), (a.errorest, b.errorest)


def test_noalloc_matches_workspace_path_two_calls_in_a_row(pg):
    w = config_workloads()["product_peak_d3"]
    cases = [
        (w.dim, w.family, w.params, w.epsrel, w.max_regions),
        (4, 1, draw_params(1, 4, 77), 1e-6, 150_000),
    ]
    for dim, fam, params, tau, cap in cases:
        a = pg.pagani_integrate_noalloc(dim, fam, params, tau, 1e-20, cap)
        b = pg.pagani_integrate_ex(dim, fam, params, tau, 1e-20, cap, relerr_filter=0 if fam == 2 else 1)
        same_result(a, b)
        assert a.n_regions > 0 and a.kernel_launches >= 4


def test_noalloc_refuses_beyond_its_capacity(pg):
    params = draw_params(1, 8, 5)
    with pytest.raises(pg.PaganiError, match="allocation-free capacity"):
        pg.pagani_integrate_noalloc(8, 1, params, 1e-6, 1e-20, 10_000_000)
    r = pg.pagani_integrate_noalloc(8, 1, params, 1e-6, 1e-20, 10_000_000, raise_on_error=False)
    assert r.status == -7
