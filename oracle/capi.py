"""ctypes front end of the C oracle (oracle/pagani_oracle.c).

ORACLE / TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke()
and the CPU-baseline leg of bench.py, never by the product package.  The
oracle is built from source with gcc (-O2 -ffp-contract=off) into
oracle/_build/; build() does that and is also called by __graft_entry__.build().
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

from . import rule as _rule
from . import rule_gm7 as _rule_gm7

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pagani_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle.so")
# The same source built with -fopenmp: only the per-region Evaluate loop of
# oracle_pagani runs in parallel (for the parallel CPU baseline).
_LIB_OMP = os.path.join(_OUT_DIR, "liboracle_omp.so")

STATUS = {0: "converged", 1: "it_max or no region left active", 2: "memory exhausted"}


def build(force: bool = False, parallel: bool = False) -> str:
    os.makedirs(_OUT_DIR, exist_ok=True)
    lib = _LIB_OMP if parallel else _LIB
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(_SRC):
        tmp = lib + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math"] +
                              (["-fopenmp"] if parallel else []) +
                              ["-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, lib)
    return lib


class _Rule(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("G", ctypes.c_int),
                ("gen", ctypes.POINTER(ctypes.c_double)), ("wts", ctypes.POINTER(ctypes.c_double)),
                ("a", ctypes.c_double), ("b", ctypes.c_double), ("q", ctypes.c_double),
                ("count", ctypes.POINTER(ctypes.c_int64)), ("error_kind", ctypes.c_int)]


class _Opt(ctypes.Structure):
    _fields_ = [("relerr_filter", ctypes.c_int), ("heuristic_filter", ctypes.c_int),
                ("init_div", ctypes.c_int), ("it_max", ctypes.c_int),
                ("lower", ctypes.c_void_p), ("upper", ctypes.c_void_p)]


class _Res(ctypes.Structure):
    _fields_ = [("estimate", ctypes.c_double), ("errorest", ctypes.c_double),
                ("status", ctypes.c_int), ("iterations", ctypes.c_int),
                ("n_regions", ctypes.c_int64), ("n_active_last", ctypes.c_int64)]


TRACE_DTYPE = np.dtype([("it", np.int32), ("trigger", np.int32), ("probes", np.int32), ("search_ok", np.int32),
                        ("s", np.int64), ("n_relerr_active", np.int64), ("n_survivors", np.int64),
                        ("v", np.float64), ("e", np.float64), ("vf", np.float64), ("ef", np.float64),
                        ("threshold", np.float64), ("direction_changes", np.float64)])

_libs: dict = {}


def _load(parallel: bool = False):
    if parallel not in _libs:
        lib = ctypes.CDLL(build(parallel=parallel))
        lib.oracle_evaluate.restype = ctypes.c_int
        lib.oracle_pagani.restype = ctypes.c_int
        lib.oracle_default_init_div.restype = ctypes.c_int
        _libs[parallel] = lib
    return _libs[parallel]


_rule_cache: dict = {}


# families whose split-axis fourth difference takes the two inner radii
# (kinks and jumps); every other family takes the inner and outer radius
_INNER_SPLIT_FAMILIES = (4, 5)   # C0, discontinuous


def split_outer(family: int) -> bool:
    return family not in _INNER_SPLIT_FAMILIES


def _rule_struct(n: int, degree: int = 9, outer: bool = True):
    """The rule as the C oracle reads it: degree 9 (the PAGANI rule, four
    null rules; outer selects the fourth difference's radii) or 7 (the
    Genz-Malik rule, error |R7 - R5|, its own radii)."""
    key = (n, degree, bool(outer) if degree == 9 else True)
    if key not in _rule_cache:
        if degree == 9:
            gen, wts = _rule.rule_tables(n)
            a, b = _rule.fourth_difference_offsets(outer)
            q = float(_rule.fourth_difference_weight(outer))
            _, counts, _, _, _ = _rule.exact_rule(n)
            kind = 0
        elif degree == 7:
            gen, wts = _rule_gm7.rule_tables(n)
            a, b, q = _rule_gm7.fourth_difference_offsets()
            _, counts, _, _, _ = _rule_gm7.exact_rule(n)
            kind = 1
        else:
            raise ValueError("rule degree must be 9 or 7")
        g = np.ascontiguousarray(gen, dtype=np.float64)
        w = np.ascontiguousarray(wts, dtype=np.float64)
        c = np.ascontiguousarray(counts, dtype=np.int64)
        r = _Rule(n, g.shape[0], g.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                  w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), a, b, q,
                  c.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), kind)
        _rule_cache[key] = (r, g, w, c)
    return _rule_cache[key][0]


def _dp(x):
    return x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def default_init_div(n: int) -> int:
    return _load().oracle_default_init_div(n)


def evaluate(family: int, n: int, params, lower, width, diag: bool = False, degree: int = 9):
    """Evaluate regions (arrays m x n).  Returns V, E (null-rule error, before
    the two-level refinement) and K; with diag=True also the diagnostic rows
    [N_1..N_4, rounding scales of N_1..N_4, rounding scale of V, D_0..D_{n-1},
    rounding scales of D_j, noise floors of N_1..N_4]."""
    lib = _load()
    lo = np.ascontiguousarray(lower, dtype=np.float64).reshape(-1, n)
    wd = np.ascontiguousarray(width, dtype=np.float64).reshape(-1, n)
    m = lo.shape[0]
    p = np.ascontiguousarray(params, dtype=np.float64)
    V = np.zeros(m)
    E = np.zeros(m)
    K = np.zeros(m, dtype=np.int32)
    D = np.zeros((m, 13 + 2 * n)) if diag else None
    lib.oracle_evaluate(ctypes.byref(_rule_struct(n, degree, split_outer(family))), ctypes.c_int(family), _dp(p), ctypes.c_int64(m),
                        _dp(lo), _dp(wd), _dp(V), _dp(E), K.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                        _dp(D) if diag else None)
    return (V, E, K, D) if diag else (V, E, K)


@dataclass
class OracleResult:
    estimate: float
    errorest: float
    status: int
    iterations: int
    n_regions: int
    n_active_last: int
    trace: np.ndarray
    final_lower: np.ndarray | None
    final_width: np.ndarray | None
    finished_volume: float
    leaves: tuple | None = None


def integrate(family: int, n: int, params, epsrel: float, epsabs: float = 1e-20, max_regions: int = 10 ** 6,
              relerr_filter: int = 1, heuristic_filter: int = 1, init_div: int = 0, it_max: int = 100,
              want_regions: bool = False, want_leaves: bool = False, bounds=None, degree: int = 9,
              parallel: bool = False) -> OracleResult:
    """bounds: None for the unit cube, else (a, b), each of length n; degree:
    the rule (9, or 7 for the Genz-Malik variant); parallel: the OpenMP
    build (per-region Evaluate on all host cores, same results)."""
    lib = _load(parallel)
    p = np.ascontiguousarray(params, dtype=np.float64)
    opt = _Opt(relerr_filter, heuristic_filter, init_div, it_max, None, None)
    if bounds is not None:
        ba = np.ascontiguousarray(bounds[0], dtype=np.float64)
        bb = np.ascontiguousarray(bounds[1], dtype=np.float64)
        assert ba.shape == (n,) and bb.shape == (n,)
        opt.lower, opt.upper = ba.ctypes.data, bb.ctypes.data
    res = _Res()
    trace = np.zeros(it_max, dtype=TRACE_DTYPE)
    fl = fw = None
    cap = 0
    if want_regions:
        cap = max_regions
        fl = np.zeros((cap, n))
        fw = np.zeros((cap, n))
    fv = ctypes.c_double(0.0)
    nleaf = ctypes.c_int64(0)
    ll = lw = None
    lcap = 0
    if want_leaves:
        lcap = 8 * max_regions
        ll = np.zeros((lcap, n))
        lw = np.zeros((lcap, n))
    lib.oracle_pagani(ctypes.byref(_rule_struct(n, degree, split_outer(family))), ctypes.c_int(family), _dp(p), ctypes.c_double(epsrel),
                      ctypes.c_double(epsabs), ctypes.c_int64(max_regions), ctypes.byref(opt), ctypes.byref(res),
                      trace.ctypes.data_as(ctypes.c_void_p), ctypes.c_int(it_max),
                      _dp(fl) if want_regions else None, _dp(fw) if want_regions else None,
                      ctypes.c_int64(cap), ctypes.byref(fv), _dp(ll) if want_leaves else None,
                      _dp(lw) if want_leaves else None, ctypes.c_int64(lcap), ctypes.byref(nleaf))
    it = res.iterations
    tr = trace[:max(it, 0)].copy()
    if want_regions:
        m = int(tr["s"][-1]) if len(tr) else 0
        fl, fw = fl[:m].copy(), fw[:m].copy()
    leaves = None
    if want_leaves:
        k = nleaf.value
        if k > lcap:
            raise RuntimeError("oracle leaf list overflow")
        leaves = (ll[:k].copy(), lw[:k].copy())
    return OracleResult(res.estimate, res.errorest, res.status, it, res.n_regions, res.n_active_last, tr,
                        fl, fw, fv.value, leaves)


def threshold_classify(A, E, v_tot: float, e_f: float, e_it: float, tau_rel: float):
    """Run the oracle's Threshold-Classify on given lists (v_tot = v + v_f,
    e_f the error finished earlier, e_it = sum E); returns
    (ok, A_out, probes, t, direction_changes)."""
    lib = _load()
    a = np.ascontiguousarray(A, dtype=np.uint8).copy()
    e = np.ascontiguousarray(E, dtype=np.float64)
    probes = ctypes.c_int(0)
    chg = ctypes.c_int(0)
    t = ctypes.c_double(0.0)
    ok = lib.oracle_threshold_classify(a.ctypes.data_as(ctypes.c_void_p), _dp(e), ctypes.c_double(v_tot),
                                       ctypes.c_double(e_f), ctypes.c_double(e_it), ctypes.c_int64(len(e)),
                                       ctypes.c_double(tau_rel), ctypes.byref(probes), ctypes.byref(t),
                                       ctypes.byref(chg))
    return ok, a, probes.value, t.value, chg.value


def gradient(family: int, n: int, params, lower, width):
    """Sum over the boxes (m x n arrays) of the basic rule applied to f and
    to df/dparams: returns (value, gradient[2n], abs_scales[2n + 1])."""
    lib = _load()
    lo = np.ascontiguousarray(lower, dtype=np.float64).reshape(-1, n)
    wd = np.ascontiguousarray(width, dtype=np.float64).reshape(-1, n)
    p = np.ascontiguousarray(params, dtype=np.float64)
    out = np.zeros(2 * n + 1)
    ab = np.zeros(2 * n + 1)
    lib.oracle_gradient(ctypes.byref(_rule_struct(n)), ctypes.c_int(family), _dp(p), ctypes.c_int64(lo.shape[0]),
                        _dp(lo), _dp(wd), _dp(out), _dp(ab))
    return out[0], out[1:], ab
