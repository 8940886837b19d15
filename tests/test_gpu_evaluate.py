"""GPU parity of Evaluate (Sec. 3.2) through the C ABI pagani_evaluate against
the oracle on identical region lists: rule value V, null-rule values N_k,
error E, fourth differences D_j and split axis K, for all seven families and
n = 2..8, with ragged counts, sibling pairs and a large list sampled."""
import numpy as np
import pytest

from oracle import capi as oracle
from paper_2104_06494_gb300.workloads import draw_params, random_dyadic_regions, SplitMix64
from tests.conftest import has_gpu
from oracle import rule as orule, rule_gm7
from tests.gpu_util import EPS, V_ROUND, null_error, sibling_regions, sum_tolerance, value_condition

pytestmark = pytest.mark.gpu

FAMS = [0, 1, 2, 3, 4, 5, 6]


@pytest.fixture(scope="module")
def torch_cuda():
    if not has_gpu():
        pytest.skip("no CUDA device")
    import torch
    import paper_2104_06494_gb300 as pg
    pg.load()
    return torch


def oracle_side(family, n, params, lo, wd, degree=9):
    Vo, Eo, Ko, Do = oracle.evaluate(family, n, params, lo, wd, diag=True, degree=degree)
    k_rel, k_abs = value_condition(family, n, params, lo, wd)
    rmod = orule if degree == 9 else rule_gm7
    _, wts = rmod.rule_tables(n)
    _, counts, _, _, _ = rmod.exact_rule(n)
    W = np.abs(np.array(wts)).T @ np.array(counts, dtype=np.float64)   # sum_g |w_gk| cnt_g, k = 0..4
    vol = np.prod(np.atleast_2d(wd), axis=1)
    # rounding floor of V: 16 u vol sum_g |w_g| M_g, M_g = |S_g| = sum_orbit |f|
    # for the positive families (the oracle's Vabs), the orbit size for the
    # oscillatory one (|f| <= 1)
    vround = V_ROUND * (vol * W[0] if family == 2 else Do[:, 8])
    return dict(V=Vo, E=Eo, K=Ko, N=Do[:, 0:4], Nabs=Do[:, 4:8], Vabs=Do[:, 8], Dj=Do[:, 9:9 + n],
                Dabs=Do[:, 9 + n:9 + 2 * n], floor=Do[:, 9 + 2 * n:13 + 2 * n], k_rel=k_rel, k_abs=k_abs,
                W=W, vol=vol, width=np.atleast_2d(wd), degree=degree, vround=vround,
                # the fourth difference's weight for this family's radii
                q=float(orule.fourth_difference_weight(oracle.split_outer(family))) if degree == 9 else 1 / 7)


def run_both(torch, family, n, params, lo, wd, degree=9):
    import paper_2104_06494_gb300 as pg
    lo_t = torch.tensor(lo.T.copy(), dtype=torch.float64, device="cuda")
    wd_t = torch.tensor(wd.T.copy(), dtype=torch.float64, device="cuda")
    V, E, K, D = pg.pagani_evaluate(n, family, params, lo_t, wd_t, diag=True, rule_degree=degree)
    torch.cuda.synchronize()
    g = dict(V=V.cpu().numpy(), E=E.cpu().numpy(), K=K.cpu().numpy(), D=D.cpu().numpy())
    return g, oracle_side(family, n, params, lo, wd, degree)


def check_parity(g, o, n):
    """Element-wise parity with tolerances derived from the arithmetic
    (tests/gpu_util.py): 1e-12 relative plus the rounding bound of each sum."""
    m = len(o["V"])
    kr, ka, vol = o["k_rel"], o["k_abs"], o["vol"]
    tolV = 1e-12 * np.abs(o["V"]) + sum_tolerance(n, o["Vabs"], kr, vol * o["W"][0], ka)
    assert np.all(np.abs(g["V"] - o["V"]) <= tolV), np.max(np.abs(g["V"] - o["V"]) / tolV)
    Ng = g["D"][0:4].T
    Fg = g["D"][4:8].T
    tolN = np.stack([1e-12 * o["N"][:, k] + sum_tolerance(n, o["Nabs"][:, k], kr, vol * o["W"][1 + k], ka)
                     for k in range(4)], axis=1)
    assert np.all(np.abs(Ng - o["N"]) <= tolN), np.max(np.abs(Ng - o["N"]) / tolN)
    # the floors are the same rounding scale on both sides
    assert np.all(np.abs(Fg - o["floor"]) <= 1e-6 * o["floor"] + tolN)
    # the kernel's E follows the error formula applied to its own floored N_k
    # (the degree-7 rule: E = |R7 - R5| = the floored N_1 itself), never
    # below the rounding floor of V (the same scale on both sides up to the
    # rounding of its own sum)
    for i in range(m):
        nu = [0.0 if Ng[i, k] <= Fg[i, k] else Ng[i, k] for k in range(4)]
        ref = null_error(*nu) if o["degree"] == 9 else nu[0]
        vr = o["vround"][i]
        tol = 1e-13 * abs(ref) + 1e-12 * vr + 1e-300
        assert abs(g["E"][i] - max(ref, vr)) <= tol, (i, g["E"][i], ref, vr)
    if o["degree"] == 7:
        assert np.all(Ng[:, 1:] == 0) and np.all(Fg[:, 1:] == 0)
    # and equals the oracle's E within the perturbation bound of the formula:
    # with N_k known to relative delta, r is known to 2 delta and
    # 10 r max(N1, r N2) to about 5 delta, so E to within 8 delta, except
    # next to the jump at r = 1, a null-value floor or the floor of V
    checked = 0
    for i in range(m):
        Nk = o["N"][i]
        if o["E"][i] <= 2 * o["vround"][i]:
            continue
        if o["degree"] == 7:
            if Nk[0] <= 4 * o["floor"][i][0] + 4 * tolN[i][0]:
                continue
            checked += 1
            assert abs(g["E"][i] - o["E"][i]) <= tolN[i][0] + 1e-12 * o["E"][i], (i, g["E"][i], o["E"][i])
            continue
        if np.any(Nk <= 4 * o["floor"][i] + 4 * tolN[i]):
            continue
        delta = float(np.max(tolN[i] / Nk))
        r = max(Nk[0] / Nk[1], Nk[1] / Nk[2], Nk[2] / Nk[3])
        if delta > 1e-3 or abs(r - 1) <= 10 * delta:
            continue
        checked += 1
        assert abs(g["E"][i] - o["E"][i]) <= (8 * delta + 1e-12) * o["E"][i], (i, g["E"][i], o["E"][i], delta)
    Dg = g["D"][8:8 + n].T
    q = o["q"]
    tolD = 1e-12 * o["Dj"] + (2 * n + 16 + kr[:, None]) * EPS * o["Dabs"] + (4 + 4 * q) * ka[:, None] * EPS
    assert np.all(np.abs(Dg - o["Dj"]) <= tolD), np.max(np.abs(Dg - o["Dj"]) / tolD)
    # split axis: equal, or a valid choice under the rounding of D and of
    # its noise floor 2^-41 M_j (M_j the magnitude sum of the five values)
    bad = np.nonzero(g["K"] != o["K"])[0]
    for i in bad:
        Dj, tj, Fj = o["Dj"][i], tolD[i], 2.0 ** -41 * o["Dabs"][i]
        sure = Dj - tj > Fj * (1 + 1e-12)
        maybe = Dj + tj > Fj * (1 - 1e-12)
        kg = g["K"][i]
        wd = o["width"][i]
        if not sure.any() and kg == int(np.argmax(wd)):
            continue                      # every difference may be at its floor
        assert maybe[kg], (i, kg, o["K"][i])
        lo_max = np.max(np.where(sure, Dj - tj, 0.0))
        hi_max = np.max(np.where(maybe, Dj + tj, 0.0))
        assert Dj[kg] + tj[kg] >= (1 - 1e-10) * lo_max, (i, kg, o["K"][i])
        assert np.all(~sure[:kg] | (Dj[:kg] - tj[:kg] < (1 - 1e-10) * hi_max)), (i, kg, o["K"][i])
    return checked


@pytest.mark.parametrize("family", FAMS)
@pytest.mark.parametrize("n", [2, 3, 4, 5, 6, 7, 8])
def test_evaluate_random_boxes(torch_cuda, family, n):
    m = 301 if n < 7 else 97          # odd: a ragged tail and an unpaired last box
    params = draw_params(family, n, 1000 + 10 * family + n)
    lo, wd = random_dyadic_regions(n, m, 77 + n, max_level=8)
    g, o = run_both(torch_cuda, family, n, params, np.array(lo), np.array(wd))
    check_parity(g, o, n)


@pytest.mark.parametrize("family", FAMS)
@pytest.mark.parametrize("n", [2, 5, 8])
def test_evaluate_sibling_pairs(torch_cuda, family, n):
    """Pairs sharing all axes but one exercise the shared factor table."""
    params = draw_params(family, n, 2000 + 10 * family + n)
    lo, wd = sibling_regions(n, 128 if n < 8 else 64, 5 + n)
    g, o = run_both(torch_cuda, family, n, params, lo, wd)
    check_parity(g, o, n)


def test_evaluate_single_and_empty(torch_cuda):
    import paper_2104_06494_gb300 as pg
    torch = torch_cuda
    params = draw_params(1, 3, 5)
    lo = np.array([[0.25, 0.5, 0.0]])
    wd = np.array([[0.25, 0.5, 1.0]])
    g, o = run_both(torch, 1, 3, params, lo, wd)
    check_parity(g, o, 3)
    z = torch.zeros((3, 0), dtype=torch.float64, device="cuda")
    V, E, K = pg.pagani_evaluate(3, 1, params, z, z)
    assert V.numel() == 0


@pytest.mark.parametrize("family,n", [(1, 5), (2, 6), (3, 8), (4, 8), (5, 6), (6, 8)])
def test_evaluate_large_list_sampled(torch_cuda, family, n):
    """A list of 2^20 boxes (many blocks, grid-stride loop) evaluated on the
    GPU; 400 sampled boxes checked against the oracle one by one."""
    import paper_2104_06494_gb300 as pg
    torch = torch_cuda
    m = 1 << 20
    gen = torch.Generator(device="cpu").manual_seed(11 + family)
    lvl = torch.randint(0, 12, (n, m), generator=gen)
    k = (torch.rand((n, m), generator=gen, dtype=torch.float64) * (2.0 ** lvl)).floor()
    wd = (0.5 ** lvl.double())
    lo = k * wd
    params = draw_params(family, n, 3000 + family)
    V, E, K, D = pg.pagani_evaluate(n, family, params, lo.cuda(), wd.cuda(), diag=True)
    rng = SplitMix64(9 + family)
    idx = sorted({int(rng.uniform(0, m)) for _ in range(400)})
    g = dict(V=V.cpu().numpy()[idx], E=E.cpu().numpy()[idx], K=K.cpu().numpy()[idx], D=D.cpu().numpy()[:, idx])
    lo_s, wd_s = lo.T.numpy()[idx], wd.T.numpy()[idx]
    check_parity(g, oracle_side(family, n, params, lo_s, wd_s), n)


@pytest.mark.parametrize("family", FAMS)
@pytest.mark.parametrize("n", [2, 3, 5, 8])
def test_evaluate_gm7_random_boxes(torch_cuda, family, n):
    """The Genz-Malik degree-7 variant: V, the difference |R7 - R5|, the
    fourth differences at its radii and the split axis against the oracle."""
    m = 301 if n < 7 else 97
    params = draw_params(family, n, 5000 + 10 * family + n)
    lo, wd = random_dyadic_regions(n, m, 97 + n, max_level=8)
    g, o = run_both(torch_cuda, family, n, params, np.array(lo), np.array(wd), degree=7)
    check_parity(g, o, n)


@pytest.mark.parametrize("family", [1, 2])
def test_evaluate_gm7_sibling_pairs(torch_cuda, family):
    n = 6
    params = draw_params(family, n, 5100 + family)
    lo, wd = sibling_regions(n, 128, 11)
    g, o = run_both(torch_cuda, family, n, params, lo, wd, degree=7)
    check_parity(g, o, n)
