"""CPU FP64 oracle -- test infrastructure only.

Only the test-suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg may import this package. It shares no code with the CUDA path
(``paper_1509_08863_gb300``) and never imports it.

The arithmetic lives in ``oracle.c`` (plain C, double precision,
single-threaded); this module compiles it with gcc on first use and wraps it
with numpy arrays. Each wrapper repeats the paper passage its C function
follows. Parity status:

* csr_build, strength, lanczos_max, cheb_coeffs, jackson, cheb_filter,
  moments, eigencount, features, cheb_filter_backward: pinned (CPU tests).
* dichotomy: pinned (exact counts with the identity as the signal block
  against a bisection on the dense spectrum).
* kmeans: pinned (brute-force argmin, numpy means, separated clusters,
  monotone inertia, ties).
* normalize (+ cheb_filter on its result): pinned (closed-form normalised
  spectra, the null vector, the dense spectral polynomial).
* adjusted_rand, stability, cheb_order: pinned (brute-force pair counting;
  gamma peaking at the true k; numpy's chebval on the same grid).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_OMP_LIB_PATH = os.path.join(_HERE, "liboracle_omp.so")
_lib = None
_omp_lib = None
_lock = threading.Lock()

_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_f32p = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")


def _compile(path: str, extra, force: bool) -> str:
    if force or not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(_SRC):
        tmp = path + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-fPIC", "-shared", "-std=c99", "-fno-fast-math"] + extra + ["-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, path)
    return path


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, -O2, IEEE semantics)."""
    return _compile(_LIB_PATH, [], force)


def build_parallel(force: bool = False) -> str:
    """The same source built with -fopenmp (liboracle_omp.so): the filter's
    loops over rows and elements run on all the threads OpenMP is given, each
    element computed exactly as in the plain build. For the timed CPU
    baseline only."""
    return _compile(_OMP_LIB_PATH, ["-fopenmp"], force)


def _load(parallel: bool = False):
    global _lib, _omp_lib
    with _lock:
        if parallel and _omp_lib is not None:
            return _omp_lib
        if not parallel and _lib is not None:
            return _lib
        lib = C.CDLL(build_parallel() if parallel else build())
        lib.oracle_threads.restype = C.c_int32
        lib.oracle_threads.argtypes = []
        lib.oracle_csr_build.restype = C.c_int64
        lib.oracle_csr_build.argtypes = [C.c_int32, C.c_int64, _i32p, _i32p, _f64p, _i32p, _i32p, _f64p]
        lib.oracle_strength.restype = None
        lib.oracle_strength.argtypes = [C.c_int32, _i32p, _i32p, _f64p, _f64p]
        lib.oracle_tridiag_max_eig.restype = C.c_double
        lib.oracle_tridiag_max_eig.argtypes = [C.c_int, _f64p, _f64p]
        lib.oracle_lanczos_max.restype = C.c_double
        lib.oracle_lanczos_max.argtypes = [C.c_int32, _i32p, _i32p, _f64p, C.c_int32, _f64p, _f64p, _f64p,
                                           C.POINTER(C.c_int32)]
        lib.oracle_jackson.restype = None
        lib.oracle_jackson.argtypes = [C.c_int32, _f64p]
        lib.oracle_cheb_coeffs.restype = None
        lib.oracle_cheb_coeffs.argtypes = [C.c_double, C.c_double, C.c_int32, C.c_int32, _f64p]
        lib.oracle_cheb_filter.restype = None
        lib.oracle_cheb_filter.argtypes = [C.c_int32, _i32p, _i32p, _f64p, C.c_double, C.c_int32, C.c_int32,
                                           _f64p, C.c_int64, _f64p, _f64p]
        lib.oracle_moments.restype = None
        lib.oracle_moments.argtypes = [C.c_int32, _i32p, _i32p, _f64p, C.c_double, C.c_int64, _f64p,
                                       C.c_int32, _f64p]
        lib.oracle_eigencount.restype = None
        lib.oracle_eigencount.argtypes = [C.c_int32, _i32p, _i32p, _f64p, C.c_double, C.c_int32, C.c_int32,
                                          _f64p, C.c_int64, _f64p, _f64p]
        lib.oracle_dichotomy.restype = C.c_double
        lib.oracle_dichotomy.argtypes = [C.c_int32, _i32p, _i32p, _f64p, C.c_double, C.c_int32, C.c_int32,
                                         C.c_int64, _f64p, C.c_double, C.c_int32, C.c_double]
        lib.oracle_features.restype = None
        lib.oracle_features.argtypes = [C.c_int32, C.c_int64, _f64p, C.c_int32, _f64p]
        lib.oracle_normalize.restype = None
        lib.oracle_normalize.argtypes = [C.c_int32, _i32p, _i32p, _f64p, _f64p, _f64p]
        lib.oracle_cheb_filter_diag.restype = None
        lib.oracle_cheb_filter_diag.argtypes = [C.c_int32, _i32p, _i32p, _f64p, _f64p, C.c_double, C.c_int32,
                                                C.c_int32, _f64p, C.c_int64, _f64p, _f64p]
        lib.oracle_adjusted_rand.restype = C.c_double
        lib.oracle_adjusted_rand.argtypes = [C.c_int32, _i32p, _i32p, C.c_int32, C.c_int32]
        lib.oracle_stability.restype = None
        lib.oracle_stability.argtypes = [C.c_int32, _i32p, _i32p, _f64p, C.c_double, C.c_int32, C.c_int32, C.c_int64,
                                         _f64p,
                                         C.c_int32, _f64p, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_uint64,
                                         _f64p, _f64p]
        lib.oracle_stability_init_row.restype = C.c_int32
        lib.oracle_stability_init_row.argtypes = [C.c_uint64, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32]
        lib.oracle_cheb_order.restype = C.c_int32
        lib.oracle_cheb_order.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int32, C.c_int32]
        lib.oracle_kmeans.restype = C.c_double
        lib.oracle_kmeans.argtypes = [C.c_int32, C.c_int32, C.c_int32, _f32p, _f32p, C.c_int32, _i32p,
                                      C.POINTER(C.c_int32)]
        lib.oracle_cheb_filter_backward.restype = None
        lib.oracle_cheb_filter_backward.argtypes = [C.c_int32, _i32p, _i32p, _f64p, C.c_double, C.c_int32,
                                                    _f64p, C.c_int64, _f64p, _f64p, _f64p, _f64p, C.c_void_p]
        if parallel:
            _omp_lib = lib
        else:
            _lib = lib
        return lib


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


class CSR:
    """Symmetric CSR of W: rowptr int32[n+1], colidx int32[nnz], val float64[nnz];
    `diag` (float64[n]) replaces the row sums as the diagonal of L when set
    (the normalised Laplacian)."""

    def __init__(self, n, rowptr, colidx, val, diag=None):
        self.n = int(n)
        self.rowptr = rowptr
        self.colidx = colidx
        self.val = val
        self.diag = diag

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def args(self):
        return self.n, self.rowptr, self.colidx, self.val


def csr_build(n, src, dst, w=None) -> CSR:
    """§2 / §2.1: symmetric W, self-loops dropped, repeated pairs merged by max."""
    lib = _load()
    src = _c(src, np.int32)
    dst = _c(dst, np.int32)
    m = src.shape[0]
    w = np.ones(m) if w is None else _c(np.asarray(w, dtype=np.float64), np.float64)
    rowptr = np.zeros(n + 1, dtype=np.int32)
    colidx = np.zeros(max(2 * m, 1), dtype=np.int32)
    val = np.zeros(max(2 * m, 1), dtype=np.float64)
    nnz = lib.oracle_csr_build(n, m, src, dst, w, rowptr, colidx, val)
    if nnz == -1:
        raise ValueError("edge endpoint outside [0, n)")
    if nnz == -2:
        raise ValueError("negative or non-finite edge weight")
    return CSR(n, rowptr, colidx[:nnz].copy(), val[:nnz].copy())


def strength(g: CSR) -> np.ndarray:
    """§2.1: s_i = sum_{j != i} W_ij."""
    s = np.zeros(g.n)
    _load().oracle_strength(g.n, g.rowptr, g.colidx, g.val, s)
    return s


def tridiag_max_eig(a, b) -> float:
    a = _c(a, np.float64)
    b = _c(b if len(b) else [0.0], np.float64)
    return _load().oracle_tridiag_max_eig(len(a), a, b)


def lanczos_max(g: CSR, iters: int, v0) -> float:
    """Largest Ritz value of L after `iters` Lanczos steps (full re-orthogonalisation)."""
    v0 = _c(v0, np.float64)
    k = C.c_int32(0)
    al = np.zeros(iters + 1)
    be = np.zeros(iters + 1)
    th = _load().oracle_lanczos_max(g.n, g.rowptr, g.colidx, g.val, iters, v0, al, be, C.byref(k))
    return th


def lambda_hat(theta_max: float, s: np.ndarray) -> float:
    """Reading of §4.1 step 1: lam_hat = min(1.01 * theta_max, 2 * max_i s_i).

    The Ritz value approaches lambda_N from below; the 1% margin keeps the
    spectrum of Lt inside [-1, 1]. 2 max_i s_i bounds lambda_N from above
    (Gershgorin). An edgeless graph gets 1.
    """
    gers = 2.0 * float(np.max(s)) if len(s) else 0.0
    lh = min(1.01 * theta_max, gers)
    return lh if lh > 0 else 1.0


def jackson(p: int) -> np.ndarray:
    g = np.zeros(p + 1)
    _load().oracle_jackson(p, g)
    return g


def cheb_coeffs(lam_max: float, cutoffs, p: int, jackson: bool = True) -> np.ndarray:
    """Chebyshev coefficients of the ideal low-pass (2), one row per cutoff."""
    cut = np.atleast_1d(np.asarray(cutoffs, dtype=np.float64))
    out = np.zeros((cut.shape[0], p + 1))
    lib = _load()
    for q, lc in enumerate(cut):
        row = np.zeros(p + 1)
        lib.oracle_cheb_coeffs(lam_max, float(lc), p, int(bool(jackson)), row)
        out[q] = row
    return out


def cheb_filter(g: CSR, lam_max: float, coeffs, R, parallel: bool = False) -> np.ndarray:
    """Y_q = sum_j a_qj T_j(Lt) R for every coefficient row q (3)/(6)/(11).
    parallel=True runs the same loops from the OpenMP build (identical results)."""
    a = np.atleast_2d(_c(coeffs, np.float64))
    a = _c(a, np.float64)
    R = _c(R, np.float64)
    n_cut, p1 = a.shape
    n, n_sig = R.shape
    Y = np.zeros((n_cut, n, n_sig))
    if g.diag is None:
        _load(parallel).oracle_cheb_filter(g.n, g.rowptr, g.colidx, g.val, lam_max, n_cut, p1 - 1, a, n_sig, R, Y)
    else:
        _load().oracle_cheb_filter_diag(g.n, g.rowptr, g.colidx, g.val, _c(g.diag, np.float64), lam_max, n_cut,
                                        p1 - 1, a, n_sig, R, Y)
    return Y


def threads(parallel: bool = False) -> int:
    """Threads the filter's loops use in the plain (1) or the OpenMP build."""
    return int(_load(parallel).oracle_threads())


def normalize(g: CSR) -> CSR:
    """The normalised Laplacian I - S^{-1/2} W S^{-1/2} (footnote of §2.1) as
    weights w_ij / sqrt(s_i s_j) and an explicit unit diagonal (0 for isolated
    nodes)."""
    val = np.zeros_like(g.val)
    diag = np.zeros(g.n)
    _load().oracle_normalize(g.n, g.rowptr, g.colidx, _c(g.val, np.float64), val, diag)
    return CSR(g.n, g.rowptr, g.colidx, val, diag)


def moments(g: CSR, lam_max: float, R, m_max: int) -> np.ndarray:
    """mu_m = <R, T_m(Lt) R> for m = 0..m_max, each from its own block."""
    R = _c(R, np.float64)
    mu = np.zeros(m_max + 1)
    _load().oracle_moments(g.n, g.rowptr, g.colidx, g.val, lam_max, R.shape[1], R, m_max, mu)
    return mu


def eigencount(g: CSR, lam_max: float, coeffs, R) -> np.ndarray:
    """§3.2 eigenvalue count per coefficient row: ||F R||_F^2."""
    a = _c(np.atleast_2d(coeffs), np.float64)
    R = _c(R, np.float64)
    out = np.zeros(a.shape[0])
    _load().oracle_eigencount(g.n, g.rowptr, g.colidx, g.val, lam_max, a.shape[0], a.shape[1] - 1, a,
                              R.shape[1], R, out)
    return out


def dichotomy(g: CSR, lam_max: float, p: int, R, k: float, jackson: bool = True, max_iter: int = 40,
              tol: float = 1e-9) -> float:
    """§3.2 dichotomy: smallest cutoff in [0, lam_max] whose count reaches k."""
    R = _c(R, np.float64)
    return _load().oracle_dichotomy(g.n, g.rowptr, g.colidx, g.val, lam_max, p, int(bool(jackson)),
                                    R.shape[1], R, float(k), max_iter, tol)


def features(Y, normalize: bool = True) -> np.ndarray:
    """Rows of the filtered block (6)/(11), optionally L2-normalised."""
    Y = _c(Y, np.float64)
    n, n_sig = Y.shape
    F = np.zeros_like(Y)
    _load().oracle_features(n, n_sig, Y, int(bool(normalize)), F)
    return F


def cheb_filter_backward(g: CSR, lam_max: float, coeffs, R, G, want_grad_R: bool = False):
    """Reverse mode of <G, sum_j a_j T_j(Lt) R>: (grad_val[nnz], grad_a[p+1], grad_R or None)."""
    a = _c(np.ravel(coeffs), np.float64)
    R = _c(R, np.float64)
    G = _c(G, np.float64)
    p = a.shape[0] - 1
    gv = np.zeros(max(g.nnz, 1))
    ga = np.zeros(p + 1)
    gR = np.zeros_like(R) if want_grad_R else None
    _load().oracle_cheb_filter_backward(
        g.n, g.rowptr, g.colidx, g.val, lam_max, p, a, R.shape[1], R, G, gv, ga,
        gR.ctypes.data if gR is not None else None)
    return gv[: g.nnz], ga, gR


def count_from_moments(mu, coeffs) -> np.ndarray:
    """count = sum_{j,j'} a_j a_j' (mu_{j+j'} + mu_{|j-j'|}) / 2, per coefficient row.

    The product rule T_j T_j' = (T_{j+j'} + T_{|j-j'|}) / 2 turns ||F R||^2
    into moments of R; the oracle uses it only to cross-check its own direct
    count (both need mu up to 2p).
    """
    a = np.atleast_2d(np.asarray(coeffs, dtype=np.float64))
    mu = np.asarray(mu, dtype=np.float64)
    p = a.shape[1] - 1
    out = np.zeros(a.shape[0])
    for q in range(a.shape[0]):
        s = 0.0
        for j in range(p + 1):
            for jj in range(p + 1):
                s += a[q, j] * a[q, jj] * 0.5 * (mu[j + jj] + mu[abs(j - jj)])
        out[q] = s
    return out


def kmeans(F, C0, max_iter: int):
    """Lloyd's k-means (§4.1 step 6, Euclidean distance between feature rows)
    from the initial centroids C0 (k x d): returns (labels int32[n], centroids
    float32[k x d], assignments performed, inertia of the last assignment).
    Distances are FP32 sums of fused multiply-adds in index order (the
    precision in which the GPU takes the same decision), ties to the lowest
    centroid; centroid means are FP64 sums in row order, rounded to FP32."""
    lib = _load()
    F = np.ascontiguousarray(F, dtype=np.float32)
    cent = np.array(C0, dtype=np.float32, copy=True, order="C")
    n, d = F.shape
    k = cent.shape[0]
    assert cent.shape[1] == d
    labels = np.full(n, -1, np.int32)
    iters = C.c_int32(0)
    inertia = lib.oracle_kmeans(n, d, k, F, cent, int(max_iter), labels, C.byref(iters))
    return labels, cent, iters.value, inertia


def adjusted_rand(a, b) -> float:
    """Adjusted Rand index of two labelings (§4.3 uses it in Eq. (12))."""
    a = _c(a, np.int32)
    b = _c(b, np.int32)
    return _load().oracle_adjusted_rand(len(a), a, b, int(a.max()) + 1, int(b.max()) + 1)


def stability(g: CSR, lam_max: float, p: int, Rc, R_blocks, kmin: int, kmax: int, max_iter: int, seed: int,
              starts: int = 1, p_filter: int | None = None):
    """gamma(k) of §4.3 / Eq. (12) for k = kmin..kmax (and the lam_k used):
    J = len(R_blocks) realisations of the filtered signals, count probes Rc,
    k-means from `starts` seeded starts per clustering (lowest inertia kept).
    The count uses order p, the filters order p_filter (None: p)."""
    Rc = _c(Rc, np.float64)
    R = _c(np.stack(R_blocks), np.float64)
    J, n, eta = R.shape
    K = kmax - kmin + 1
    gamma = np.zeros(K)
    lam_k = np.zeros(K)
    pf = int(p) if p_filter is None else int(p_filter)
    _load().oracle_stability(g.n, g.rowptr, g.colidx, g.val, lam_max, p, pf, eta, Rc, J, R, kmin, kmax, max_iter,
                             int(starts), int(seed), gamma, lam_k)
    return gamma, lam_k


def stability_init_row(seed: int, j: int, k: int, t: int, c: int, n: int) -> int:
    return _load().oracle_stability_init_row(int(seed), j, k, t, c, n)


def cheb_order(x: float, delta: float, w: float, jackson: bool = True, p_max: int = 1000) -> int:
    """m*(lambda_c / lambda_N; delta) of §2.4 with the band |t - x| < w left out
    (-1 when no order up to p_max meets delta)."""
    return _load().oracle_cheb_order(float(x), float(delta), float(w), int(bool(jackson)), int(p_max))
