"""GB300-native PAGANI adaptive integration (Sakiotis et al., SC'21).

Thin ctypes binding of the C ABI in include/pagani.h (argument marshalling
only): every step of the integration runs in the CUDA kernels of
libpagani_gb300.so.  There is no CPU fallback: if the library is missing or
cannot be loaded, every call raises.

PyTorch is used, where a caller wants it, only for device memory and streams
(``evaluate`` accepts CUDA tensors).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

PRODUCT_PEAK, GAUSSIAN, OSCILLATORY, CORNER_PEAK, C0, DISCONTINUOUS, BOX_POWER = 0, 1, 2, 3, 4, 5, 6
STATUS_NAMES = {0: "converged", 1: "it_max or no region left", 2: "memory exhausted",
                -1: "bad dim", -2: "bad integrand", -3: "bad tolerance", -4: "cuda error", -5: "watchdog",
                -6: "non-finite integrand", -7: "capacity below initial split", -8: "bad argument"}

LIB_PATH = _build.LIB


class PaganiError(RuntimeError):
    pass


class Result(ctypes.Structure):
    _fields_ = [("estimate", ctypes.c_double), ("errorest", ctypes.c_double), ("status", ctypes.c_int32),
                ("iterations", ctypes.c_int32), ("n_regions", ctypes.c_int64), ("n_active_last", ctypes.c_int64),
                ("finished_volume", ctypes.c_double), ("eval_ms", ctypes.c_double), ("eval_launches", ctypes.c_int32),
                ("kernel_launches", ctypes.c_int32), ("h2d_bytes", ctypes.c_int64), ("d2h_bytes", ctypes.c_int64),
                ("active_volume", ctypes.c_double), ("n_leaves", ctypes.c_int64),
                ("phase_ms", ctypes.c_double * 4)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class BatchItem(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("integrand_id", ctypes.c_int32), ("relerr_filter", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("epsrel", ctypes.c_double), ("epsabs", ctypes.c_double),
                ("params", ctypes.c_double * 17)]


class BatchResult(ctypes.Structure):
    _fields_ = [("estimate", ctypes.c_double), ("errorest", ctypes.c_double), ("status", ctypes.c_int32),
                ("iterations", ctypes.c_int32), ("n_regions", ctypes.c_int64)]


class Options(ctypes.Structure):
    _fields_ = [("relerr_filter", ctypes.c_int32), ("heuristic_filter", ctypes.c_int32),
                ("init_div", ctypes.c_int32), ("it_max", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("keep_leaves", ctypes.c_int32), ("rule_degree", ctypes.c_int32)]


TRACE_DTYPE = np.dtype([("it", np.int32), ("trigger", np.int32), ("probes", np.int32), ("search_ok", np.int32),
                        ("s", np.int64), ("n_relerr_active", np.int64), ("n_survivors", np.int64),
                        ("v", np.float64), ("e", np.float64), ("vf", np.float64), ("ef", np.float64),
                        ("threshold", np.float64), ("direction_changes", np.float64),
                        ("probe_passes", np.int32), ("reserved", np.int32)])

# every symbol include/pagani.h declares
EXPORTED = ["pagani_default_options", "pagani_integrate", "pagani_integrate_ex", "pagani_workspace_reserve",
            "pagani_workspace_release", "pagani_evaluate", "pagani_rule_tables", "pagani_fp64_peak",
            "pagani_last_error", "pagani_version", "pagani_integrate_noalloc", "pagani_leaves", "pagani_gradient",
            "pagani_integrate_batch", "pagani_integrate_box", "pagani_evaluate_ex",
            "pagani_rule_tables_ex"]

_lib = None


def load(build_if_missing: bool = False) -> ctypes.CDLL:
    """Loads libpagani_gb300.so (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        if not build_if_missing:
            raise PaganiError(f"{LIB_PATH} is missing: run paper_2104_06494_gb300.build.build() first")
        _build.build()
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    lib.pagani_default_options.argtypes = [P(Options)]
    lib.pagani_default_options.restype = None
    lib.pagani_integrate.argtypes = [ctypes.c_int, ctypes.c_int, P(ctypes.c_double), ctypes.c_double,
                                     ctypes.c_double, ctypes.c_int64, P(Result)]
    lib.pagani_integrate.restype = ctypes.c_int
    lib.pagani_integrate_ex.argtypes = [ctypes.c_int, ctypes.c_int, P(ctypes.c_double), ctypes.c_double,
                                        ctypes.c_double, ctypes.c_int64, P(Options), ctypes.c_void_p, P(Result),
                                        ctypes.c_void_p, ctypes.c_int]
    lib.pagani_integrate_ex.restype = ctypes.c_int
    lib.pagani_integrate_box.argtypes = [ctypes.c_int, ctypes.c_int, P(ctypes.c_double), P(ctypes.c_double),
                                         P(ctypes.c_double), ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                         P(Options), ctypes.c_void_p, P(Result), ctypes.c_void_p, ctypes.c_int]
    lib.pagani_integrate_box.restype = ctypes.c_int
    lib.pagani_integrate_noalloc.argtypes = [ctypes.c_int, ctypes.c_int, P(ctypes.c_double), ctypes.c_double,
                                             ctypes.c_double, ctypes.c_int64, ctypes.c_void_p, P(Result)]
    lib.pagani_integrate_noalloc.restype = ctypes.c_int
    lib.pagani_workspace_reserve.argtypes = [ctypes.c_int64, ctypes.c_int]
    lib.pagani_workspace_reserve.restype = ctypes.c_int
    lib.pagani_workspace_release.argtypes = []
    lib.pagani_workspace_release.restype = ctypes.c_int
    lib.pagani_evaluate.argtypes = [ctypes.c_int, ctypes.c_int, P(ctypes.c_double), ctypes.c_int64,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.pagani_evaluate.restype = ctypes.c_int
    lib.pagani_evaluate_ex.argtypes = [ctypes.c_int, ctypes.c_int, P(ctypes.c_double), ctypes.c_int, ctypes.c_int64,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.pagani_evaluate_ex.restype = ctypes.c_int
    lib.pagani_leaves.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, P(ctypes.c_int64),
                                  ctypes.c_void_p]
    lib.pagani_leaves.restype = ctypes.c_int
    lib.pagani_gradient.argtypes = [ctypes.c_int, ctypes.c_int, P(ctypes.c_double), ctypes.c_int64, ctypes.c_void_p,
                                    ctypes.c_void_p, P(ctypes.c_double), ctypes.c_void_p]
    lib.pagani_gradient.restype = ctypes.c_int
    lib.pagani_integrate_batch.argtypes = [ctypes.c_int64, P(BatchItem), ctypes.c_int64, P(Options), ctypes.c_void_p,
                                           P(BatchResult), P(ctypes.c_double)]
    lib.pagani_integrate_batch.restype = ctypes.c_int
    lib.pagani_rule_tables.argtypes = [ctypes.c_int, P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_int64)]
    lib.pagani_rule_tables.restype = ctypes.c_int
    lib.pagani_rule_tables_ex.argtypes = [ctypes.c_int, ctypes.c_int, P(ctypes.c_double), P(ctypes.c_double),
                                          P(ctypes.c_int64)]
    lib.pagani_rule_tables_ex.restype = ctypes.c_int
    lib.pagani_fp64_peak.argtypes = [P(ctypes.c_double), ctypes.c_int, ctypes.c_void_p]
    lib.pagani_fp64_peak.restype = ctypes.c_int
    lib.pagani_last_error.argtypes = []
    lib.pagani_last_error.restype = ctypes.c_char_p
    lib.pagani_version.argtypes = []
    lib.pagani_version.restype = ctypes.c_char_p
    _lib = lib
    return lib


def last_error() -> str:
    return load().pagani_last_error().decode()


def _params_array(params):
    p = np.ascontiguousarray(params, dtype=np.float64)
    return p, p.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def default_options() -> Options:
    o = Options()
    load().pagani_default_options(ctypes.byref(o))
    return o


@dataclass
class Integration:
    estimate: float
    errorest: float
    status: int
    iterations: int
    n_regions: int
    n_active_last: int
    finished_volume: float
    eval_ms: float = -1.0
    eval_launches: int = 0
    kernel_launches: int = 0
    h2d_bytes: int = 0
    d2h_bytes: int = 0
    trace: np.ndarray | None = None
    active_volume: float = 0.0
    n_leaves: int = -1
    phase_ms: tuple = (-1.0, -1.0, -1.0, -1.0)   # fill, probe, count, split (host-driven loop)

    @property
    def status_name(self) -> str:
        return STATUS_NAMES.get(self.status, str(self.status))


def _integration(r: Result, trace=None) -> Integration:
    return Integration(r.estimate, r.errorest, r.status, r.iterations, r.n_regions, r.n_active_last,
                       r.finished_volume, r.eval_ms, r.eval_launches, r.kernel_launches, r.h2d_bytes, r.d2h_bytes,
                       trace, r.active_volume, r.n_leaves, tuple(r.phase_ms))


def pagani_integrate(dim: int, integrand_id: int, params, epsrel: float, epsabs: float = 1e-20,
                     max_regions: int = 10_000_000) -> Integration:
    """C ABI pagani_integrate (default options, library stream)."""
    lib = load()
    p, pp = _params_array(params)
    r = Result()
    rc = lib.pagani_integrate(dim, integrand_id, pp, epsrel, epsabs, max_regions, ctypes.byref(r))
    if rc < 0:
        raise PaganiError(f"pagani_integrate failed ({rc}): {last_error()}")
    return _integration(r)


def pagani_integrate_ex(dim: int, integrand_id: int, params, epsrel: float, epsabs: float = 1e-20,
                        max_regions: int = 10_000_000, relerr_filter: int = 1, heuristic_filter: int = 1,
                        init_div: int = 0, it_max: int = 100, use_graph: int = 1, stream: int | None = None,
                        trace: bool = False, raise_on_error: bool = True, keep_leaves: int = 0,
                        bounds=None, rule_degree: int = 9) -> Integration:
    """C ABI pagani_integrate_ex, or pagani_integrate_box when bounds = (a, b)
    (each of length dim) is given; stream is a raw cudaStream_t (e.g.
    torch.cuda.current_stream().cuda_stream) or None for the library stream."""
    lib = load()
    p, pp = _params_array(params)
    o = Options(relerr_filter, heuristic_filter, init_div, it_max, use_graph, keep_leaves, rule_degree)
    r = Result()
    tr = np.zeros(it_max, dtype=TRACE_DTYPE) if trace else None
    tail = (ctypes.byref(o), ctypes.c_void_p(stream or 0), ctypes.byref(r),
            tr.ctypes.data_as(ctypes.c_void_p) if trace else None, it_max if trace else 0)
    if bounds is None:
        name = "pagani_integrate_ex"
        rc = lib.pagani_integrate_ex(dim, integrand_id, pp, epsrel, epsabs, max_regions, *tail)
    else:
        name = "pagani_integrate_box"
        a, pa = _params_array(bounds[0])
        b, pb = _params_array(bounds[1])
        if a.shape != (dim,) or b.shape != (dim,):
            raise ValueError("bounds must be two arrays of length dim")
        rc = lib.pagani_integrate_box(dim, integrand_id, pp, pa, pb, epsrel, epsabs, max_regions, *tail)
    if rc < 0 and raise_on_error:
        raise PaganiError(f"{name} failed ({rc}): {last_error()}")
    if trace:
        tr = tr[:max(min(r.iterations, it_max), 0)].copy()
    return _integration(r, tr)


def pagani_integrate_noalloc(dim: int, integrand_id: int, params, epsrel: float, epsabs: float = 1e-20,
                             max_regions: int = 100_000, stream: int | None = None,
                             raise_on_error: bool = True) -> Integration:
    """C ABI pagani_integrate_noalloc: the allocation-free integration for
    callers that cannot allocate device memory (see include/pagani.h)."""
    lib = load()
    p, pp = _params_array(params)
    r = Result()
    rc = lib.pagani_integrate_noalloc(dim, integrand_id, pp, epsrel, epsabs, max_regions,
                                      ctypes.c_void_p(stream or 0), ctypes.byref(r))
    if rc < 0 and raise_on_error:
        raise PaganiError(f"pagani_integrate_noalloc failed ({rc}): {last_error()}")
    return _integration(r)


def pagani_workspace_reserve(max_regions: int, dim: int) -> None:
    rc = load().pagani_workspace_reserve(max_regions, dim)
    if rc < 0:
        raise PaganiError(f"pagani_workspace_reserve failed ({rc}): {last_error()}")


def pagani_workspace_release() -> None:
    load().pagani_workspace_release()


def pagani_evaluate(dim: int, integrand_id: int, params, lower, width, diag: bool = False, stream: int | None = None,
                    rule_degree: int = 9):
    """Evaluate on caller boxes (C ABI pagani_evaluate_ex).  lower, width:
    CUDA tensors (float64) of shape (dim, m) (SoA).  Returns CUDA tensors V,
    E (float64), K (int32) and, with diag=True, the (8 + dim, m) diagnostics
    (N_1..N_4, their noise floors, D_j)."""
    import torch

    lib = load()
    if lower.dtype != torch.float64 or width.dtype != torch.float64 or not lower.is_cuda or not width.is_cuda:
        raise PaganiError("lower and width must be float64 CUDA tensors")
    lower = lower.contiguous()
    width = width.contiguous()
    m = lower.shape[1]
    dev = lower.device
    V = torch.empty(m, dtype=torch.float64, device=dev)
    E = torch.empty(m, dtype=torch.float64, device=dev)
    K = torch.empty(m, dtype=torch.int32, device=dev)
    D = torch.empty((8 + dim, m), dtype=torch.float64, device=dev) if diag else None
    p, pp = _params_array(params)
    if stream is None:
        stream = torch.cuda.current_stream(dev).cuda_stream
    rc = lib.pagani_evaluate_ex(dim, integrand_id, pp, rule_degree, m, ctypes.c_void_p(lower.data_ptr()),
                                ctypes.c_void_p(width.data_ptr()), ctypes.c_void_p(V.data_ptr()),
                                ctypes.c_void_p(E.data_ptr()), ctypes.c_void_p(K.data_ptr()),
                                ctypes.c_void_p(D.data_ptr()) if diag else None, ctypes.c_void_p(stream))
    if rc < 0:
        raise PaganiError(f"pagani_evaluate failed ({rc}): {last_error()}")
    return (V, E, K, D) if diag else (V, E, K)


def pagani_leaves(dim: int, stream: int | None = None):
    """The leaf set kept by the last integration with keep_leaves=1, as CUDA
    tensors lower (dim, m) float64 and level (dim, m) uint8."""
    import torch

    lib = load()
    n = ctypes.c_int64(0)
    rc = lib.pagani_leaves(dim, 0, None, None, ctypes.byref(n), None)
    if rc < 0:
        raise PaganiError(f"pagani_leaves failed ({rc}): {last_error()}")
    m = n.value
    lower = torch.empty((dim, m), dtype=torch.float64, device="cuda")
    level = torch.empty((dim, m), dtype=torch.uint8, device="cuda")
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    rc = lib.pagani_leaves(dim, m, ctypes.c_void_p(lower.data_ptr()), ctypes.c_void_p(level.data_ptr()),
                           ctypes.byref(n), ctypes.c_void_p(stream))
    if rc < 0:
        raise PaganiError(f"pagani_leaves failed ({rc}): {last_error()}")
    return lower, level


def pagani_gradient(dim: int, integrand_id: int, params, lower, level, stream: int | None = None):
    """(value, gradient) of the rule estimate over the boxes (lower, level)
    (CUDA tensors of shape (dim, m)); gradient in the params layout."""
    import torch

    lib = load()
    p, pp = _params_array(params)
    lower = lower.contiguous()
    level = level.contiguous()
    out = np.zeros(2 * dim + 1)
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    rc = lib.pagani_gradient(dim, integrand_id, pp, lower.shape[1], ctypes.c_void_p(lower.data_ptr()),
                             ctypes.c_void_p(level.data_ptr()), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                             ctypes.c_void_p(stream))
    if rc < 0:
        raise PaganiError(f"pagani_gradient failed ({rc}): {last_error()}")
    return out[0], out[1:]


def pagani_integrate_batch(items, max_regions_per_item: int, heuristic_filter: int = 1, it_max: int = 100,
                           use_graph: int = 1, stream: int | None = None):
    """C ABI pagani_integrate_batch.  items: sequence of Workload-like objects
    (dim, family, params, epsrel, epsabs, relerr_filter).  Returns (numpy
    structured results in item order, device milliseconds of the loop)."""
    lib = load()
    n = len(items)
    arr = (BatchItem * n)()
    for i, w in enumerate(items):
        arr[i].dim = w.dim
        arr[i].integrand_id = w.family
        arr[i].relerr_filter = w.relerr_filter
        arr[i].epsrel = w.epsrel
        arr[i].epsabs = w.epsabs
        for k, v in enumerate(w.params):
            arr[i].params[k] = v
    res = (BatchResult * n)()
    o = Options(1, heuristic_filter, 0, it_max, use_graph, 0)
    ms = ctypes.c_double(0.0)
    rc = lib.pagani_integrate_batch(n, arr, max_regions_per_item, ctypes.byref(o), ctypes.c_void_p(stream or 0), res,
                                    ctypes.byref(ms))
    if rc < 0:
        raise PaganiError(f"pagani_integrate_batch failed ({rc}): {last_error()}")
    out = np.zeros(n, dtype=[("estimate", np.float64), ("errorest", np.float64), ("status", np.int32),
                             ("iterations", np.int32), ("n_regions", np.int64)])
    for i in range(n):
        out[i] = (res[i].estimate, res[i].errorest, res[i].status, res[i].iterations, res[i].n_regions)
    return out, ms.value


def pagani_rule_tables(dim: int, rule_degree: int = 9):
    """(num_points, radius[5], weights[9, 5], counts[9]) as generated by the
    library (host code), for the degree-9 rule or the degree-7 variant."""
    lib = load()
    rad = np.zeros(5)
    w = np.zeros(45)
    cnt = np.zeros(9, dtype=np.int64)
    npts = lib.pagani_rule_tables_ex(dim, rule_degree, rad.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                     w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                     cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    if npts < 0:
        raise PaganiError(f"pagani_rule_tables failed ({npts}): {last_error()}")
    return npts, rad, w.reshape(9, 5), cnt


def pagani_fp64_peak(stream: int | None = None) -> dict:
    """Measured FP64 throughput: FMA TFLOP/s and exp, sincos, division rates (1e9/s)."""
    out = (ctypes.c_double * 4)()
    rc = load().pagani_fp64_peak(out, 4, ctypes.c_void_p(stream or 0))
    if rc < 0:
        raise PaganiError(f"pagani_fp64_peak failed ({rc}): {last_error()}")
    return {"fma_tflops": out[0], "exp_gps": out[1], "sincos_gps": out[2], "div_gps": out[3]}


def version() -> str:
    return load().pagani_version().decode()
