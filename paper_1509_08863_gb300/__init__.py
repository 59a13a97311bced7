"""GB300 graph filtering of random signals for accelerated spectral clustering.

Thin Python binding over the C ABI of ``libspecfilt.so`` (declared in
``include/specfilt.h``). Every step of the path runs in the library's CUDA
kernels; this module only marshals arguments: PyTorch supplies device memory
and the current CUDA stream, numpy carries small host tables (coefficients,
moments, counts).

The library must be built (``paper_1509_08863_gb300.build.build()``); if it
is missing every call raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

__all__ = [
    "SpecFiltError",
    "Opts",
    "Graph",
    "Batch",
    "lib",
    "csr_build",
    "lambda_max_estimate",
    "cheb_coeffs",
    "cheb_filter",
    "cheb_moments",
    "cheb_moments_noalloc",
    "count_from_moments",
    "eigencount",
    "eigencount_from",
    "dichotomy",
    "features",
    "row_sumsq",
    "features_scaled",
    "cheb_filter_backward",
    "batch_build",
    "cheb_filter_batched",
    "cheb_filter_batched_dev",
    "autotune",
    "profile_begin",
    "profile_end",
    "profile_variants",
    "launch_count",
    "device_check",
    "ChebFilter",
    "F32",
    "BF16",
    "F16",
    "ALGO_AUTO",
    "ALGO_FORWARD",
    "ALGO_CLENSHAW",
]

F32, BF16, F16 = 0, 1, 2
ALGO_AUTO, ALGO_FORWARD, ALGO_CLENSHAW = 0, 1, 2
SWEEP_AUTO, SWEEP_TILED, SWEEP_DIRECT, SWEEP_PERSISTENT = 0, 1, 2, 3
HINTS_NONE, HINT_IDX_EVICT_FIRST, HINT_OUT_STREAMING, HINT_MIXED_ADD = -1, 1, 2, 8

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libspecfilt.so")
_lib = None


class SpecFiltError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        self.status = status
        super().__init__(f"{where}: status {status}: {detail}")


class _Opts(C.Structure):
    _fields_ = [
        ("storage", C.c_int32),
        ("algo", C.c_int32),
        ("slab_cols", C.c_int32),
        ("block_warps", C.c_int32),
        ("blocks_per_sm", C.c_int32),
        ("ckpt_every", C.c_int32),
        ("mem_cap_mb", C.c_int64),
        ("carveout_pct", C.c_int32),
        ("l2_window", C.c_int32),
        ("sweep_kernel", C.c_int32),
        ("sweep_hints", C.c_int32),
    ]


@dataclass
class Opts:
    """Mirror of ``sf_opts`` (zeros mean automatic)."""

    storage: int = F32
    algo: int = ALGO_AUTO
    slab_cols: int = 0
    block_warps: int = 0
    blocks_per_sm: int = 0
    ckpt_every: int = 0
    mem_cap_mb: int = 0
    carveout_pct: int = 0
    l2_window: int = 0
    sweep_kernel: int = 0
    sweep_hints: int = 0

    def c(self) -> _Opts:
        return _Opts(self.storage, self.algo, self.slab_cols, self.block_warps, self.blocks_per_sm,
                      self.ckpt_every, self.mem_cap_mb, self.carveout_pct, self.l2_window, self.sweep_kernel,
                      self.sweep_hints)


_vp = C.c_void_p
_i32 = C.c_int32
_i64 = C.c_int64
_f64 = C.c_double
_dp = C.POINTER(C.c_double)


def lib():
    """Load libspecfilt.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise SpecFiltError(-1, "load", f"{LIB_PATH} is missing; build it with paper_1509_08863_gb300.build.build()")
    L = C.CDLL(LIB_PATH)
    sig = {
        "sf_status_str": (C.c_char_p, [_i32]),
        "sf_last_error": (C.c_char_p, []),
        "sf_version": (_i32, []),
        "sf_launch_count": (_i64, []),
        "sf_csr_build": (_i32, [_i32, _i64, _vp, _vp, _vp, _vp, C.POINTER(_vp)]),
        "sf_graph_info": (_i32, [_vp, C.POINTER(_i32), C.POINTER(_i64), C.POINTER(_i32), _dp]),
        "sf_graph_csr": (_i32, [_vp, C.POINTER(_vp), C.POINTER(_vp), C.POINTER(_vp), C.POINTER(_vp)]),
        "sf_graph_set_values": (_i32, [_vp, _vp, _vp]),
        "sf_graph_free": (None, [_vp]),
        "sf_lambda_max_estimate": (_i32, [_vp, _i32, _vp, C.c_uint64, _vp, _dp, _dp]),
        "sf_cheb_coeffs": (_i32, [_f64, _dp, _i32, _i32, _i32, _dp]),
        "sf_cheb_filter": (_i32, [_vp, _f64, _dp, _i32, _i32, _vp, _i32, _i32, _vp, C.POINTER(_Opts), _vp]),
        "sf_cheb_moments": (_i32, [_vp, _f64, _vp, _i32, _i32, _i32, _dp, C.POINTER(_Opts), _vp]),
        "sf_count_from_moments": (_i32, [_dp, _i32, _dp, _i32, _dp]),
        "sf_eigencount": (_i32, [_vp, _f64, _vp, _i32, _i32, _i32, _dp, _i32, _i32, _dp, _dp, C.POINTER(_Opts),
                                 _vp]),
        "sf_dichotomy": (_i32, [_dp, _i32, _f64, _f64, _i32, _i32, _f64, _dp]),
        "sf_features": (_i32, [_vp, _i32, _i32, _i32, _vp, _vp]),
        "sf_row_sumsq": (_i32, [_vp, _i32, _i32, _vp, _vp]),
        "sf_features_scaled": (_i32, [_vp, _i32, _i32, _vp, _vp, _vp]),
        "sf_cheb_filter_backward": (_i32, [_vp, _f64, _dp, _i32, _vp, _i32, _vp, _vp, _dp, _vp,
                                           C.POINTER(_Opts), _vp]),
        "sf_batch_build": (_i32, [C.POINTER(_vp), _i32, _vp, C.POINTER(_vp)]),
        "sf_batch_info": (_i32, [_vp, C.POINTER(_i32), C.POINTER(_i64), C.POINTER(_i32), C.POINTER(_i32)]),
        "sf_batch_free": (None, [_vp]),
        "sf_cheb_filter_batched": (_i32, [_vp, _dp, _dp, _i32, _vp, _i32, _i32, _vp, C.POINTER(_Opts), _vp]),
        "sf_cheb_filter_batched_dev": (_i32, [_vp, _vp, _vp, _i32, _vp, _i32, _i32, _vp, C.POINTER(_Opts), _vp]),
        "sf_cheb_filter_batched_multi": (_i32, [_vp, _dp, _dp, _i32, _i32, _vp, _i32, _i32, _vp, C.POINTER(_Opts),
                                                _vp]),
        "sf_autotune": (_i32, [_vp, _i32, _i32, _i32, C.POINTER(_Opts), _vp, C.POINTER(_Opts)]),
        "sf_profile_begin": (_i32, []),
        "sf_device_check": (_i32, [_vp]),
        "sf_cheb_moments_noalloc": (_i32, [_vp, _f64, _vp, _i32, _i32, _dp, _vp]),
        "sf_profile_end": (_i32, [C.POINTER(_i64), _dp, _dp]),
        "sf_profile_variant": (_i32, [_i32, C.POINTER(_i64), _dp, _dp]),
        "sf_kmeans": (_i32, [_vp, _i32, _i32, _i32, _vp, _i32, _i32, _vp, C.POINTER(_i32), _dp, _vp]),
        "sf_graph_normalize": (_i32, [_vp, _vp, C.POINTER(_vp)]),
        "sf_adjusted_rand": (_i32, [_vp, _vp, _i32, _i32, _i32, _vp, _dp]),
        "sf_stability": (_i32, [_vp, _f64, _i32, _i32, _vp, _vp, _i32, _i32, _i32, _i32, _i32, _i32, C.c_uint64, _vp,
                                _vp, _dp, _dp, C.POINTER(_i32)]),
        "sf_cheb_order": (_i32, [_f64, _f64, _f64, _i32, _i32, C.POINTER(_i32)]),
        "sf_selftest_bounded_wait": (_i32, [_i32, _vp]),
        "sf_selftest_arrival_wait": (_i32, [_i32, _vp]),
        "sf_gather_ceiling": (_i32, [_i64, _i32, _i32, _i32, _vp, _dp]),
        "sf_gather_rate": (_i32, [_i64, _i32, _i32, _i32, _i32, _vp, _dp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(st: int, where: str):
    if st != 0:
        L = lib()
        raise SpecFiltError(st, where, L.sf_last_error().decode(errors="replace"))


def _torch():
    import torch

    return torch


def _stream():
    torch = _torch()
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev_ptr(t, dtype=None, name="tensor"):
    torch = _torch()
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return C.c_void_p(t.data_ptr())


def _f64arr(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def _rdtype(R):
    torch = _torch()
    if R.dtype == torch.float32:
        return F32
    if R.dtype == torch.bfloat16:
        return BF16
    raise TypeError(f"R must be float32 or bfloat16, got {R.dtype}")


def _opts_ptr(opts):
    if opts is None:
        return None, None
    o = opts.c() if isinstance(opts, Opts) else opts
    return o, C.byref(o)


class _DevView:
    """__cuda_array_interface__ over a borrowed device pointer."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": shape, "typestr": typestr, "data": (ptr, False), "version": 2,
                                         "strides": None}


class Graph:
    """Device CSR of W owned by the library (§2, §2.1)."""

    def __init__(self, handle: int):
        self._h = C.c_void_p(handle)

    @property
    def handle(self):
        return self._h

    def info(self):
        n, nnz, unit, smax = _i32(), _i64(), _i32(), _f64()
        _check(lib().sf_graph_info(self._h, C.byref(n), C.byref(nnz), C.byref(unit), C.byref(smax)), "sf_graph_info")
        return n.value, nnz.value, bool(unit.value), smax.value

    @property
    def n(self):
        return self.info()[0]

    @property
    def nnz(self):
        return self.info()[1]

    def csr(self):
        """Copies (torch CUDA tensors) of rowptr, colidx, val, strength."""
        torch = _torch()
        n, nnz, _, _ = self.info()
        rp, ci, va, st = _vp(), _vp(), _vp(), _vp()
        _check(lib().sf_graph_csr(self._h, C.byref(rp), C.byref(ci), C.byref(va), C.byref(st)), "sf_graph_csr")
        torch.cuda.synchronize()

        def view(ptr, shape, ts, dt):
            if shape[0] == 0 or not ptr.value:
                return torch.zeros(shape, dtype=dt, device="cuda")
            return torch.as_tensor(_DevView(ptr.value, shape, ts), device="cuda").clone()

        return (view(rp, (n + 1,), "<i4", torch.int32), view(ci, (nnz,), "<i4", torch.int32),
                view(va, (nnz,), "<f4", torch.float32), view(st, (n,), "<f8", torch.float64))

    def normalized(self) -> "Graph":
        """The normalised Laplacian I - S^-1/2 W S^-1/2 (footnote of §2.1) as a new graph."""
        out = _vp()
        _check(lib().sf_graph_normalize(self._h, _stream(), C.byref(out)), "sf_graph_normalize")
        return Graph(out.value)

    def set_values(self, val):
        torch = _torch()
        _check(lib().sf_graph_set_values(self._h, _dev_ptr(val, torch.float32, "val"), _stream()),
               "sf_graph_set_values")

    def free(self):
        if self._h is not None and self._h.value:
            lib().sf_graph_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def csr_build(n: int, src, dst, w=None) -> Graph:
    """Symmetric CSR of W from an undirected edge list (int32 src/dst, float32 w on the GPU)."""
    torch = _torch()
    m = int(src.shape[0])
    out = _vp()
    _check(lib().sf_csr_build(int(n), m, _dev_ptr(src, torch.int32, "src"), _dev_ptr(dst, torch.int32, "dst"),
                              _dev_ptr(w, torch.float32, "w") if w is not None else None, _stream(),
                              C.byref(out)), "sf_csr_build")
    return Graph(out.value)


def lambda_max_estimate(g: Graph, iters: int = 40, v0=None, seed: int = 0):
    """(theta_max, lam_hat): Lanczos Ritz value and the bound used by the filters (§4.1 step 1)."""
    torch = _torch()
    th, lh = _f64(), _f64()
    _check(lib().sf_lambda_max_estimate(g.handle, int(iters), _dev_ptr(v0, torch.float64, "v0") if v0 is not None
                                        else None, C.c_uint64(seed), _stream(), C.byref(th), C.byref(lh)),
           "sf_lambda_max_estimate")
    return th.value, lh.value


def cheb_coeffs(lam_max: float, cutoffs, p: int, jackson: bool = True) -> np.ndarray:
    cut, cp = _f64arr(np.atleast_1d(cutoffs))
    out = np.zeros((cut.shape[0], p + 1))
    _check(lib().sf_cheb_coeffs(float(lam_max), cp, cut.shape[0], int(p), int(bool(jackson)),
                                out.ctypes.data_as(_dp)), "sf_cheb_coeffs")
    return out


def cheb_filter(g: Graph, lam_max: float, coeffs, R, opts: Opts | None = None, out=None):
    """Y[c] = sum_j coeffs[c, j] T_j(Lt) R on the GPU; returns a float32 tensor [n_cut, N, n_sig]."""
    torch = _torch()
    a, ap = _f64arr(np.atleast_2d(coeffs))
    n_cut, p1 = a.shape
    n, n_sig = R.shape
    if out is None:
        out = torch.empty((n_cut, n, n_sig), dtype=torch.float32, device=R.device)
    o, op = _opts_ptr(opts)
    _check(lib().sf_cheb_filter(g.handle, float(lam_max), ap, n_cut, p1 - 1, _dev_ptr(R, None, "R"), _rdtype(R),
                                n_sig, _dev_ptr(out, torch.float32, "Y"), op, _stream()), "sf_cheb_filter")
    return out


def cheb_moments(g: Graph, lam_max: float, R, p: int, opts: Opts | None = None) -> np.ndarray:
    n, n_sig = R.shape
    mu = np.zeros(2 * p + 1)
    o, op = _opts_ptr(opts)
    _check(lib().sf_cheb_moments(g.handle, float(lam_max), _dev_ptr(R, None, "R"), _rdtype(R), n_sig, int(p),
                                 mu.ctypes.data_as(_dp), op, _stream()), "sf_cheb_moments")
    return mu


def cheb_moments_noalloc(g: Graph, lam_max: float, R, p: int) -> np.ndarray:
    """sf_cheb_moments_noalloc: the moments with no device allocation (FP32 R)."""
    torch = _torch()
    n, n_sig = R.shape
    mu = np.zeros(2 * p + 1)
    _check(lib().sf_cheb_moments_noalloc(g.handle, float(lam_max), _dev_ptr(R, torch.float32, "R"), n_sig, int(p),
                                         mu.ctypes.data_as(_dp), _stream()), "sf_cheb_moments_noalloc")
    return mu


def count_from_moments(mu, p: int, coeffs) -> np.ndarray:
    mu, mp = _f64arr(mu)
    a, ap = _f64arr(np.atleast_2d(coeffs))
    out = np.zeros(a.shape[0])
    _check(lib().sf_count_from_moments(mp, int(p), ap, a.shape[0], out.ctypes.data_as(_dp)),
           "sf_count_from_moments")
    return out


def eigencount(g: Graph, lam_max: float, R, p: int, cutoffs, jackson: bool = True, opts: Opts | None = None):
    """(counts per cutoff, moments) of §3.2 from one moment sweep."""
    n, n_sig = R.shape
    cut, cp = _f64arr(np.atleast_1d(cutoffs))
    counts = np.zeros(cut.shape[0])
    mu = np.zeros(2 * p + 1)
    o, op = _opts_ptr(opts)
    _check(lib().sf_eigencount(g.handle, float(lam_max), _dev_ptr(R, None, "R"), _rdtype(R), n_sig, int(p), cp,
                               cut.shape[0], int(bool(jackson)), counts.ctypes.data_as(_dp), mu.ctypes.data_as(_dp),
                               op, _stream()), "sf_eigencount")
    return counts, mu


def eigencount_from(mu, p: int, lam_max: float, cutoffs, jackson: bool = True) -> np.ndarray:
    """Counts of §3.2 at the given cutoffs from already computed moments (host only)."""
    return count_from_moments(mu, p, cheb_coeffs(lam_max, cutoffs, p, jackson))


def dichotomy(mu, p: int, lam_max: float, k: float, jackson: bool = True, max_iter: int = 40,
              tol: float = 1e-9) -> float:
    mu, mp = _f64arr(mu)
    out = _f64()
    _check(lib().sf_dichotomy(mp, int(p), float(lam_max), float(k), int(bool(jackson)), int(max_iter), float(tol),
                              C.byref(out)), "sf_dichotomy")
    return out.value


def features(Y, normalize: bool = True, out=None):
    torch = _torch()
    n, n_sig = Y.shape
    if out is None:
        out = torch.empty_like(Y)
    _check(lib().sf_features(_dev_ptr(Y, torch.float32, "Y"), n, n_sig, int(bool(normalize)),
                             _dev_ptr(out, torch.float32, "F"), _stream()), "sf_features")
    return out


def row_sumsq(Y, out=None):
    """Per-row sums of squares (float64 tensor) of a float32 block."""
    torch = _torch()
    n, n_sig = Y.shape
    if out is None:
        out = torch.empty(n, dtype=torch.float64, device=Y.device)
    _check(lib().sf_row_sumsq(_dev_ptr(Y, torch.float32, "Y"), n, n_sig, _dev_ptr(out, torch.float64, "sumsq"),
                              _stream()), "sf_row_sumsq")
    return out


def features_scaled(Y, sumsq, out=None):
    """Rows of Y divided by sqrt(sumsq) (sumsq summed over all column shards)."""
    torch = _torch()
    n, n_sig = Y.shape
    if out is None:
        out = torch.empty_like(Y)
    _check(lib().sf_features_scaled(_dev_ptr(Y, torch.float32, "Y"), n, n_sig,
                                    _dev_ptr(sumsq, torch.float64, "sumsq"), _dev_ptr(out, torch.float32, "F"),
                                    _stream()), "sf_features_scaled")
    return out


def cheb_filter_backward(g: Graph, lam_max: float, coeffs, R, G, want_grad_R: bool = True,
                         opts: Opts | None = None):
    """(grad_val [nnz], grad_coeffs [p+1] numpy, grad_R or None) of <G, Y>."""
    torch = _torch()
    a, ap = _f64arr(np.ravel(coeffs))
    n, n_sig = R.shape
    nnz = g.nnz
    gv = torch.empty(max(nnz, 1), dtype=torch.float32, device=R.device)
    ga = np.zeros(a.shape[0])
    gR = torch.empty_like(R) if want_grad_R else None
    o, op = _opts_ptr(opts)
    _check(lib().sf_cheb_filter_backward(g.handle, float(lam_max), ap, a.shape[0] - 1,
                                         _dev_ptr(R, torch.float32, "R"), n_sig, _dev_ptr(G, torch.float32, "G"),
                                         _dev_ptr(gv, torch.float32, "grad_val"), ga.ctypes.data_as(_dp),
                                         _dev_ptr(gR, torch.float32, "grad_R") if gR is not None else None, op,
                                         _stream()), "sf_cheb_filter_backward")
    return gv[:nnz], ga, gR


class Batch:
    """Block-diagonal concatenation of several graphs."""

    def __init__(self, handle: int):
        self._h = C.c_void_p(handle)

    @property
    def handle(self):
        return self._h

    def info(self):
        n, nnz, ng = _i32(), _i64(), _i32()
        _check(lib().sf_batch_info(self._h, C.byref(n), C.byref(nnz), C.byref(ng), None), "sf_batch_info")
        offs = (C.c_int32 * (ng.value + 1))()
        _check(lib().sf_batch_info(self._h, None, None, None, offs), "sf_batch_info")
        return n.value, nnz.value, ng.value, np.array(offs[:], dtype=np.int64)

    def free(self):
        if self._h is not None and self._h.value:
            lib().sf_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def batch_build(graphs) -> Batch:
    arr = (C.c_void_p * len(graphs))(*[g.handle.value for g in graphs])
    out = _vp()
    _check(lib().sf_batch_build(arr, len(graphs), _stream(), C.byref(out)), "sf_batch_build")
    return Batch(out.value)


def cheb_filter_batched(b: Batch, lam_max, coeffs, R, opts: Opts | None = None, out=None):
    """Every graph of the batch filtered with its own lam_max and coefficient row (one launch per order, or one
    persistent launch for all orders with opts.sweep_kernel = SWEEP_PERSISTENT)."""
    torch = _torch()
    lm, lp = _f64arr(np.ravel(lam_max))
    a, ap = _f64arr(np.atleast_2d(coeffs))
    n, n_sig = R.shape
    if out is None:
        out = torch.empty((n, n_sig), dtype=torch.float32, device=R.device)
    o, op = _opts_ptr(opts)
    _check(lib().sf_cheb_filter_batched(b.handle, lp, ap, a.shape[1] - 1, _dev_ptr(R, None, "R"), _rdtype(R), n_sig,
                                        _dev_ptr(out, torch.float32, "Y"), op, _stream()), "sf_cheb_filter_batched")
    return out


def cheb_filter_batched_multi(b: Batch, lam_max, coeffs, R, opts: Opts | None = None, out=None):
    """Every graph filtered at n_cut cutoffs: coeffs [n_graphs, n_cut, p + 1]; returns [n_cut, N, n_sig]."""
    torch = _torch()
    lm, lp = _f64arr(np.ravel(lam_max))
    a, ap = _f64arr(np.asarray(coeffs, np.float64))
    if a.ndim != 3:
        raise ValueError("coeffs must be [n_graphs, n_cut, p + 1]")
    n, n_sig = R.shape
    n_cut = a.shape[1]
    if out is None:
        out = torch.empty((n_cut, n, n_sig), dtype=torch.float32, device=R.device)
    o, op = _opts_ptr(opts)
    _check(lib().sf_cheb_filter_batched_multi(b.handle, lp, ap, n_cut, a.shape[2] - 1, _dev_ptr(R, None, "R"),
                                              _rdtype(R), n_sig, _dev_ptr(out, torch.float32, "Y"), op, _stream()),
           "sf_cheb_filter_batched_multi")
    return out


def cheb_filter_batched_dev(b: Batch, two_over_lam, coeffs, R, out, opts: Opts | None = None):
    """Batched filter with device tables (float64 2/lam per graph, float32 [graphs, p+1] coefficients):
    no host copies and no synchronisation, so it can be captured in a CUDA graph."""
    torch = _torch()
    n, n_sig = R.shape
    o, op = _opts_ptr(opts)
    _check(lib().sf_cheb_filter_batched_dev(b.handle, _dev_ptr(two_over_lam, torch.float64, "two_over_lam"),
                                            _dev_ptr(coeffs, torch.float32, "coeffs"), coeffs.shape[1] - 1,
                                            _dev_ptr(R, None, "R"), _rdtype(R), n_sig,
                                            _dev_ptr(out, torch.float32, "Y"), op, _stream()),
           "sf_cheb_filter_batched_dev")
    return out


def autotune(g: Graph, n_sig: int, storage: int = F32, n_cut: int = 1, base: Opts | None = None) -> Opts:
    b, bp = _opts_ptr(base)
    best = _Opts()
    _check(lib().sf_autotune(g.handle, int(n_sig), int(storage), int(n_cut), bp, _stream(), C.byref(best)),
           "sf_autotune")
    return Opts(best.storage, best.algo, best.slab_cols, best.block_warps, best.blocks_per_sm, best.ckpt_every,
                best.mem_cap_mb, best.carveout_pct, best.l2_window, best.sweep_kernel, best.sweep_hints)


def profile_begin():
    _check(lib().sf_profile_begin(), "sf_profile_begin")


def profile_end():
    """(launches, total ms, total algorithmic bytes) of the sweep kernel since profile_begin()."""
    n, ms, by = _i64(), _f64(), _f64()
    _check(lib().sf_profile_end(C.byref(n), C.byref(ms), C.byref(by)), "sf_profile_end")
    return n.value, ms.value, by.value


KMEANS_AUTO, KMEANS_TENSOR, KMEANS_CUDA_CORES, KMEANS_TENSOR_SINGLE = 0, 1, 2, 3


def kmeans(F, C0, max_iter: int = 50, mode: int = KMEANS_AUTO):
    """Lloyd's k-means on the rows of F (§4.1 step 6) from centroids C0 (k x d):
    returns (labels int32 tensor [n], centroids float32 tensor [k x d],
    assignments performed, inertia of the last assignment). mode:
    KMEANS_AUTO (tensor cores when the shape allows), KMEANS_TENSOR (tcgen05
    distances from split TF32 operands), KMEANS_TENSOR_SINGLE (one TF32
    product per pair) or KMEANS_CUDA_CORES; every mode returns the labels of
    the same FP32 decision."""
    torch = _torch()
    n, d = F.shape
    k = C0.shape[0]
    Fd = F.contiguous()
    Cw = C0.to(device=F.device, dtype=torch.float32).contiguous().clone()
    labels = torch.empty(n, dtype=torch.int32, device=F.device)
    it = _i32()
    inertia = _f64()
    _check(lib().sf_kmeans(_dev_ptr(Fd, torch.float32, "F"), int(n), int(d), int(k), Cw.data_ptr(), int(max_iter),
                           int(mode), labels.data_ptr(), C.byref(it), C.byref(inertia), _stream()), "sf_kmeans")
    return labels, Cw, it.value, inertia.value


def adjusted_rand(a, b, ka: int | None = None, kb: int | None = None) -> float:
    """Adjusted Rand index of two int32 label tensors on the device."""
    torch = _torch()
    ka = int(a.max().item()) + 1 if ka is None else ka
    kb = int(b.max().item()) + 1 if kb is None else kb
    r = _f64()
    _check(lib().sf_adjusted_rand(_dev_ptr(a, torch.int32, "a"), _dev_ptr(b, torch.int32, "b"), int(a.shape[0]),
                                  int(ka), int(kb), _stream(), C.byref(r)), "sf_adjusted_rand")
    return r.value


def stability(g: Graph, lam_max: float, p: int, Rc, R, kmin: int, kmax: int, max_iter: int = 50,
              starts: int = 4, seed: int = 0, opts: Opts | None = None, p_filter: int | None = None,
              return_order: bool = False):
    """gamma(k) of §4.3 / Eq. (12) for k = kmin..kmax and the lam_k used:
    count probes Rc [N, eta], realisations R [J, N, eta] (FP32, on the device).
    p: the count's order; p_filter: the filters' order (None: p; 0: the order
    at which the filters of adjacent k differ). return_order adds the order used."""
    torch = _torch()
    J, n, eta = R.shape
    K = kmax - kmin + 1
    gamma = np.zeros(K)
    lam_k = np.zeros(K)
    used = _i32()
    o, op = _opts_ptr(opts)
    pf = int(p) if p_filter is None else int(p_filter)
    _check(lib().sf_stability(g.handle, float(lam_max), int(p), pf, _dev_ptr(Rc, torch.float32, "Rc"),
                              _dev_ptr(R, torch.float32, "R"), int(J), int(eta), int(kmin), int(kmax), int(max_iter),
                              int(starts), int(seed), op, _stream(), gamma.ctypes.data_as(_dp),
                              lam_k.ctypes.data_as(_dp), C.byref(used)), "sf_stability")
    return (gamma, lam_k, used.value) if return_order else (gamma, lam_k)


def cheb_order(x: float, delta: float, w: float, jackson: bool = True, p_max: int = 1000) -> int:
    """m*(lambda_c / lambda_N; delta) of §2.4 with the band |t - x| < w left out (-1: none up to p_max)."""
    m = _i32()
    _check(lib().sf_cheb_order(float(x), float(delta), float(w), int(bool(jackson)), int(p_max), C.byref(m)),
           "sf_cheb_order")
    return m.value


def gather_ceiling(n_rows: int, row_bytes: int, deg: int, reps: int = 10) -> float:
    """Rows per second of the sweep's random-row gather pattern with each output
    row's sums written back (synthetic BF16 table of n_rows + 1 rows of
    row_bytes bytes, deg entries per row)."""
    r = _f64()
    _check(lib().sf_gather_ceiling(int(n_rows), int(row_bytes), int(deg), int(reps), _stream(), C.byref(r)),
           "sf_gather_ceiling")
    return r.value


def gather_rate(n_rows: int, row_bytes: int, deg: int, reps: int = 10, write_rows: bool = False) -> float:
    """Rows per second of the same pattern; without write_rows, the gathers alone."""
    r = _f64()
    _check(lib().sf_gather_rate(int(n_rows), int(row_bytes), int(deg), int(reps), int(bool(write_rows)), _stream(),
                                C.byref(r)), "sf_gather_rate")
    return r.value


def selftest_arrival_wait(polls: int = 1000):
    """Make the persistent batch sweep's arrival wait give up (nothing faults); the next device_check raises
    SF_ERR_TIMEOUT."""
    _check(lib().sf_selftest_arrival_wait(int(polls), _stream()), "sf_selftest_arrival_wait")


def selftest_bounded_wait(polls: int = 1000):
    """Make a kernel's bounded wait give up (nothing faults); the next device_check raises SF_ERR_TIMEOUT."""
    _check(lib().sf_selftest_bounded_wait(int(polls), _stream()), "sf_selftest_bounded_wait")


def device_check():
    """Synchronise the current stream; raise if a sweep kernel gave up a bounded wait."""
    _check(lib().sf_device_check(_stream()), "sf_device_check")


PROFILE_TAGS = {3 * m + s: f"{mn}_{sn}" for m, mn in enumerate(("forward", "moments", "clenshaw"))
                for s, sn in enumerate(("f32", "bf16", "f16"))}
PROFILE_TAGS[9] = "adjoint_f32"
PROFILE_TAGS[10] = "kmeans_tc_f32"


def profile_variants():
    """{variant name: (launches, ms, bytes)} of the last profile_end()."""
    out = {}
    for tag, name in PROFILE_TAGS.items():
        n, ms, by = _i64(), _f64(), _f64()
        _check(lib().sf_profile_variant(tag, C.byref(n), C.byref(ms), C.byref(by)), "sf_profile_variant")
        if n.value:
            out[name] = (n.value, ms.value, by.value)
    return out


def launch_count() -> int:
    return int(lib().sf_launch_count())


def _autograd():
    torch = _torch()

    class _ChebFilter(torch.autograd.Function):
        """Y = sum_j a_j T_j(Lt) R with gradients for the edge weights (CSR order),
        the coefficients and R; lam_max is held fixed."""

        @staticmethod
        def forward(ctx, val, coeffs, R, graph, lam_max, opts):
            graph.set_values(val.detach().contiguous())
            a = coeffs.detach().cpu().double().numpy()
            Y = cheb_filter(graph, lam_max, a[None, :], R.detach().contiguous(), opts)[0]
            ctx.save_for_backward(val, coeffs, R)
            ctx.graph, ctx.lam_max, ctx.opts = graph, lam_max, opts
            return Y

        @staticmethod
        def backward(ctx, G):
            val, coeffs, R = ctx.saved_tensors
            ctx.graph.set_values(val.detach().contiguous())
            a = coeffs.detach().cpu().double().numpy()
            gv, ga, gR = cheb_filter_backward(ctx.graph, ctx.lam_max, a, R.detach().contiguous(),
                                              G.contiguous().float(), want_grad_R=ctx.needs_input_grad[2],
                                              opts=ctx.opts)
            gcoef = torch.as_tensor(ga, dtype=coeffs.dtype, device=coeffs.device)
            return gv, gcoef, gR, None, None, None

    return _ChebFilter


_CF = None


def ChebFilter(val, coeffs, R, graph: Graph, lam_max: float, opts: Opts | None = None):
    """Differentiable filter: gradients flow to `val` (CSR-order weights), `coeffs` and `R`."""
    global _CF
    if _CF is None:
        _CF = _autograd()
    return _CF.apply(val, coeffs, R, graph, lam_max, opts)
