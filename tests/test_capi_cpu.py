"""CPU checks of the product library: it builds for sm_103a, loads, exports
every symbol include/pagani.h declares, generates the same rule tables as the
oracle (two independent constructions: exact rationals vs long-double least
squares), rejects invalid arguments on the host, and has no CPU fallback."""
import os
import re

import numpy as np
import pytest

import paper_2104_06494_gb300 as pg
from paper_2104_06494_gb300 import build as pbuild
from oracle import rule as orule
from tests.conftest import has_gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    pbuild.build()
    return pg.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pagani.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pagani_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    decl = declared_functions()
    assert decl, "no declarations parsed"
    assert sorted(pg.EXPORTED) == decl
    for name in decl:
        assert hasattr(lib, name), name


def test_library_is_sm103a_only():
    assert pbuild.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


@pytest.mark.parametrize("n", range(2, 9))
def test_rule_tables_match_oracle(lib, n):
    npts, rad, w, cnt = pg.pagani_rule_tables(n)
    assert npts == orule.num_points(n)
    gen, wts = orule.rule_tables(n)
    _, counts, _, _, _ = orule.exact_rule(n)
    names = orule.generator_names(n)
    full = ["centre", "l1", "l2", "l3", "lp", "l1l1", "l1l2", "l1l1l1", "l0^n"]
    # the fourth difference's radii: the l2 and l1 slots (smooth families),
    # the lp and l2 slots (families with kinks or jumps)
    a, b = orule.fourth_difference_offsets(outer=True)
    assert abs(rad[1] - a) <= 2e-16 and abs(rad[0] - b) <= 2e-16
    a, b = orule.fourth_difference_offsets(outer=False)
    assert abs(rad[3] - a) <= 1e-16 and abs(rad[1] - b) <= 2e-16
    for gi, name in enumerate(names):
        g = full.index(name)
        assert cnt[g] == counts[gi]
        for k in range(5):
            ref = wts[gi][k]
            colscale = max(abs(r[k]) for r in wts)
            # norm-wise: every entry within 1e-15 of the rule vector's scale
            # (entries that nearly cancel, and the exactly zero lambda_p basic
            # weight, are not resolved relative to themselves)
            assert abs(w[g, k] - ref) <= 1e-15 * colscale, (n, name, k, w[g, k], ref)
    # the absent triple orbit of n = 2 carries nothing
    if n == 2:
        assert cnt[7] == 0 and np.all(w[7] == 0)


@pytest.mark.parametrize("n", range(2, 9))
def test_gm7_rule_tables_match_oracle(lib, n):
    """The library's degree-7 tables (host long double, QR on closed-form
    orbit moments) against the oracle's exact rationals, slot by slot: the
    Genz-Malik orbits sit on the centre, lp (sqrt(9/70)), l2 (sqrt(9/10)),
    l1l1 (sqrt(9/10) pairs) and l0^n (sqrt(9/19)) slots; column 1 is w7 - w5."""
    from oracle import rule_gm7
    npts, rad, w, cnt = pg.pagani_rule_tables(n, rule_degree=7)
    assert npts == rule_gm7.num_points(n) == 2 ** n + 2 * n * n + 2 * n + 1
    gen, wts = rule_gm7.rule_tables(n)
    _, counts, _, _, _ = rule_gm7.exact_rule(n)
    slots = [0, 4, 2, 5, 8]
    a, b, q = rule_gm7.fourth_difference_offsets()
    assert abs(rad[3] - a) <= 1e-16 and abs(rad[1] - b) <= 2e-16 and abs(rad[0] - b) <= 2e-16
    assert abs(rad[4] - gen[4][0]) <= 2e-16
    for gi, g in enumerate(slots):
        assert cnt[g] == counts[gi]
        for k in (0, 1):
            colscale = max(abs(r[k]) for r in wts)
            assert abs(w[g, k] - wts[gi][k]) <= 1e-15 * colscale, (n, g, k, w[g, k], wts[gi][k])
    others = [g for g in range(9) if g not in slots]
    assert np.all(cnt[others] == 0) and np.all(w[others] == 0) and np.all(w[:, 2:] == 0)


def test_host_argument_checks(lib):
    with pytest.raises(pg.PaganiError):
        pg.pagani_integrate(1, 0, [1.0, 0.5], 1e-3)
    with pytest.raises(pg.PaganiError):
        pg.pagani_integrate(3, 9, [1.0] * 6, 1e-3)
    with pytest.raises(pg.PaganiError):
        pg.pagani_integrate(3, 0, [7.0] * 6, 0.0)
    with pytest.raises(pg.PaganiError):
        pg.pagani_integrate(3, 0, [0.0] * 6, 1e-3)       # product peak needs c != 0
    with pytest.raises(pg.PaganiError):
        pg.pagani_integrate(3, 0, [7.0] * 6, 1e-3, max_regions=100)  # below the initial split
    with pytest.raises(pg.PaganiError, match="-8"):
        pg.pagani_integrate_ex(3, 0, [7.0] * 6, 1e-3, heuristic_filter=4)  # trigger modes are 0..3
    with pytest.raises(pg.PaganiError, match="-8"):
        pg.pagani_integrate_ex(3, 0, [7.0] * 6, 1e-3, rule_degree=8)       # rules are 9 and 7
    with pytest.raises(pg.PaganiError, match="-8"):
        pg.pagani_integrate_ex(3, 0, [7.0] * 6, 1e-3, rule_degree=7, keep_leaves=1)
    with pytest.raises(pg.PaganiError):
        pg.pagani_rule_tables(3, rule_degree=5)
    with pytest.raises(pg.PaganiError, match="-8"):
        pg.pagani_integrate_ex(3, 0, [7.0] * 6, 1e-3, bounds=([0.0, 0.5, 0.0], [1.0, 0.5, 1.0]))  # empty box
    with pytest.raises(pg.PaganiError, match="-8"):
        pg.pagani_integrate_ex(3, 0, [7.0] * 6, 1e-3, bounds=([0.0, 0.0, -1e308], [1.0, 1.0, 1e308]))
    with pytest.raises(pg.PaganiError, match="-2"):
        pg.pagani_integrate(3, pg.BOX_POWER, [-1.0], 1e-3)                # box power needs q >= 0
    with pytest.raises(pg.PaganiError, match="-2"):
        pg.pagani_integrate(3, pg.DISCONTINUOUS, [1.0, 2.0, float("nan"), 0.5, 0.5, 0.5], 1e-3)


@pytest.mark.skipif(has_gpu(), reason="checks the behaviour without a GPU")
def test_no_cpu_fallback_without_gpu(lib):
    with pytest.raises(pg.PaganiError, match="-4"):
        pg.pagani_integrate(3, 0, [7.0, 8.0, 9.0, 0.4, 0.5, 0.6], 1e-3)
