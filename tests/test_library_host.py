"""CPU-side checks of the C-ABI library: it loads, exports every declared
entry point, and its host-only FP64 logic (coefficients, counts from
moments, dichotomy, status strings) agrees with the oracle. No GPU work."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sflib():
    from paper_1509_08863_gb300 import build

    build.build()
    import paper_1509_08863_gb300 as sf

    return sf


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"SF_API\s+[^;{(]*?\b(sf_\w+)\s*\(", txt, flags=re.S))
    return sorted(names)


def test_exports_every_declared_symbol(sflib):
    names = declared_symbols()
    assert len(names) >= 20, names
    L = C.CDLL(sflib.LIB_PATH)
    for nm in names:
        assert hasattr(L, nm), nm


def test_status_strings(sflib):
    L = sflib.lib()
    assert L.sf_status_str(0) == b"SF_OK"
    assert b"invalid argument" in L.sf_status_str(1)
    assert L.sf_version() >= 100


def test_host_coefficients_match_oracle(sflib, oracle_mod):
    for lam, cuts, p, jk in [(7.5, [0.3, 2.0, 7.5], 40, True), (1.0, [0.0, 0.5], 7, False), (3.0, [1.2], 200, True)]:
        a = sflib.cheb_coeffs(lam, cuts, p, jk)
        b = oracle_mod.cheb_coeffs(lam, cuts, p, jk)
        np.testing.assert_allclose(a, b, rtol=1e-13, atol=1e-15)


def test_host_count_from_moments_and_dichotomy(sflib, oracle_mod):
    from helpers import cliques_edges

    k, m, eta, p = 4, 7, 120, 60
    src, dst = cliques_edges(k, m)
    g = oracle_mod.csr_build(k * m, src, dst)
    lam = 1.01 * m
    R = np.random.default_rng(2).standard_normal((k * m, eta)) / np.sqrt(eta)
    mu = oracle_mod.moments(g, lam, R, 2 * p)
    a = oracle_mod.cheb_coeffs(lam, [0.5, 3.0, 6.0], p, True)
    np.testing.assert_allclose(sflib.count_from_moments(mu, p, a), oracle_mod.count_from_moments(mu, a), rtol=1e-12)
    lk = sflib.dichotomy(mu, p, lam, k - 0.5, True, 40, 1e-9)
    lo = oracle_mod.dichotomy(g, lam, p, R, k - 0.5, True, 40, 1e-9)
    assert abs(lk - lo) <= 2e-9 * lam * 4


def test_argument_errors_without_gpu(sflib):
    L = sflib.lib()
    out = np.zeros(3)
    cut = np.array([0.5])
    st = L.sf_cheb_coeffs(-1.0, cut.ctypes.data_as(C.POINTER(C.c_double)), 1, 2, 1,
                          out.ctypes.data_as(C.POINTER(C.c_double)))
    assert st == 1 and b"lam_max" in L.sf_last_error()


def test_kmeans_argument_checks_without_gpu(sflib):
    """sf_kmeans checks its arguments before any device work: bad sizes and modes, and a tensor-core request
    for a shape the tensor cores do not take, return SF_ERR_ARG with a message (the pointers are never read)."""
    L = sflib.lib()
    fake = C.c_void_p(16)  # 16-byte aligned, never dereferenced
    it = C.c_int32(0)
    iner = C.c_double(0.0)

    def call(n, d, k, max_iter, mode):
        return L.sf_kmeans(fake, n, d, k, fake, max_iter, mode, fake, C.byref(it), C.byref(iner), None)

    assert call(100, 32, 0, 10, 0) == 1 and b"k must be" in L.sf_last_error()
    assert call(0, 32, 4, 10, 0) == 1
    assert call(100, 32, 4, 0, 0) == 1 and b"max_iter" in L.sf_last_error()
    assert call(100, 32, 4, 10, 7) == 1 and b"mode" in L.sf_last_error()
    for mode in (sflib.KMEANS_TENSOR, sflib.KMEANS_TENSOR_SINGLE):
        assert call(100, 30, 4, 10, mode) == 1 and b"tensor-core" in L.sf_last_error()  # d not a multiple of 32
        assert call(100, 32, 129, 10, mode) == 1  # k > 128


def test_stability_and_rand_argument_checks_without_gpu(sflib):
    """sf_adjusted_rand and sf_stability reject bad arguments before reading any pointer or launching work."""
    L = sflib.lib()
    fake = C.c_void_p(16)
    ari = C.c_double(0.0)
    assert L.sf_adjusted_rand(None, fake, 10, 2, 2, None, C.byref(ari)) == 1
    assert L.sf_adjusted_rand(fake, fake, 0, 2, 2, None, C.byref(ari)) == 1
    assert L.sf_adjusted_rand(fake, fake, 10, 5000, 5000, None, C.byref(ari)) == 1 and b"2^24" in L.sf_last_error()
    gam = np.zeros(8)
    lk = np.zeros(8)
    dp = C.POINTER(C.c_double)

    used = C.c_int32(-7)

    def stab(J, kmin, kmax, max_iter, starts, p_filter=20):
        return L.sf_stability(fake, 10.0, 20, p_filter, fake, fake, J, 8, kmin, kmax, max_iter, starts, 1, None, None,
                              gam.ctypes.data_as(dp), lk.ctypes.data_as(dp), C.byref(used))

    assert stab(1, 2, 4, 10, 2) == 1 and b"J >= 2" in L.sf_last_error()
    assert stab(3, 5, 4, 10, 2) == 1 and b"kmin" in L.sf_last_error()
    assert stab(3, 2, 4, 0, 2) == 1 and b"max_iter" in L.sf_last_error()
    assert stab(3, 2, 4, 10, 0) == 1 and b"starts" in L.sf_last_error()
    assert stab(3, 2, 4, 10, 2, p_filter=-1) == 1 and b"p_filter" in L.sf_last_error()
    assert stab(3, 2, 4, 10, 2, p_filter=20001) == 1 and b"p_filter" in L.sf_last_error()
    assert np.all(gam == 0) and np.all(lk == 0) and used.value == -7  # outputs untouched


def test_filter_and_moment_argument_checks_without_gpu(sflib):
    """The sweeps' entry points reject a missing graph or block, a bad lam_max, order, width or dtype before
    they look at the graph or the device; the host outputs stay untouched."""
    L = sflib.lib()
    fake = C.c_void_p(16)
    dp = C.POINTER(C.c_double)
    coef = np.ones(3)
    mom = np.zeros(5)

    def filt(g, lam, p, R, dtype, n_sig):
        return L.sf_cheb_filter(g, lam, coef.ctypes.data_as(dp), 1, p, R, dtype, n_sig, fake, None, None)

    def moments(g, lam, p, R, dtype, n_sig):
        return L.sf_cheb_moments(g, lam, R, dtype, n_sig, p, mom.ctypes.data_as(dp), None, None)

    for call in (filt, moments):
        assert call(None, 10.0, 2, fake, 0, 4) == 1 and b"graph" in L.sf_last_error()
        assert call(fake, -1.0, 2, fake, 0, 4) == 1 and b"lam_max" in L.sf_last_error()
        assert call(fake, float("nan"), 2, fake, 0, 4) == 1
        assert call(fake, 10.0, -1, fake, 0, 4) == 1 and b"p must" in L.sf_last_error()
        assert call(fake, 10.0, 2, fake, 0, 0) == 1 and b"n_sig" in L.sf_last_error()
        assert call(fake, 10.0, 2, None, 0, 4) == 1 and b"R is NULL" in L.sf_last_error()
        assert call(fake, 10.0, 2, fake, 2, 4) == 1 and b"dtype" in L.sf_last_error()  # FP16 input blocks
    assert np.all(mom == 0)


def test_graph_and_feature_argument_checks_without_gpu(sflib):
    """sf_csr_build and sf_features reject bad sizes and missing buffers before any device work; the
    graph handle is cleared on failure, and an empty feature block is a no-op."""
    L = sflib.lib()
    fake = C.c_void_p(16)
    out = C.c_void_p(12345)
    assert L.sf_csr_build(0, 10, fake, fake, None, None, C.byref(out)) == 1 and out.value is None
    assert L.sf_csr_build(10, -1, fake, fake, None, None, C.byref(out)) == 1
    assert L.sf_csr_build(10, 1 << 30, fake, fake, None, None, C.byref(out)) == 1 and b"2^31" in L.sf_last_error()
    assert L.sf_csr_build(10, 5, None, fake, None, None, C.byref(out)) == 1 and b"src/dst" in L.sf_last_error()
    assert L.sf_csr_build(10, 5, fake, fake, None, None, None) == 1 and b"out is NULL" in L.sf_last_error()
    assert L.sf_features(None, 10, 4, 1, fake, None) == 1
    assert L.sf_features(fake, 10, 0, 1, fake, None) == 1 and b"n_sig" in L.sf_last_error()
    assert L.sf_features(fake, 0, 4, 1, fake, None) == 0  # nothing to do, no launch


def test_host_cheb_order_matches_oracle(sflib, oracle_mod):
    """The order table m* of §2.4 (host FP64, Clenshaw evaluation) equals the
    oracle's (direct cos(j arccos) evaluation) on a spread of cutoffs."""
    for x in (0.01, 0.05, 0.2, 0.5, 0.9):
        for delta, w in ((0.1, 0.01), (0.1, 0.05), (0.05, 0.02)):
            assert sflib.cheb_order(x, delta, w, True, 800) == oracle_mod.cheb_order(x, delta, w, True, 800)
    with pytest.raises(sflib.SpecFiltError):
        sflib.cheb_order(1.5, 0.1, 0.01)


def test_diagnostic_argument_checks_without_gpu(sflib):
    """The gather diagnostics reject bad sizes before allocating or launching anything, and leave the
    result untouched."""
    L = sflib.lib()
    r = C.c_double(-1.0)
    for args in ((0, 64, 32, 1), (1000, 48, 32, 1), (1000, 64, 30, 1), (1000, 64, 0, 1), (1000, 64, 32, 0),
                 (1 << 31, 64, 32, 1)):
        assert L.sf_gather_ceiling(*args, None, C.byref(r)) == 1
        assert L.sf_gather_rate(*args, 0, None, C.byref(r)) == 1
        assert L.sf_gather_rate(*args, 1, None, C.byref(r)) == 1
    assert r.value == -1.0
    assert L.sf_gather_rate(1000, 64, 32, 1, 0, None, None) == 1 and b"rows_per_s" in L.sf_last_error()
