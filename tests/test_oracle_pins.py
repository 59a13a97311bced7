"""Pins of the CPU oracle to things other than itself (CPU only).

Each test checks one oracle function against what the paper or mathematics
fixes: brute force on tiny inputs, closed forms, a dense eigendecomposition,
quadrature, finite differences, statistical expectations. A plausible slip in
the oracle (dropped term, wrong sign or index, transposed operand) fails at
least one of them.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate

from helpers import cheb_eval, cliques_edges, dense_laplacian, dense_w, random_graph

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def to_dense(g):
    W = np.zeros((g.n, g.n))
    for i in range(g.n):
        for e in range(g.rowptr[i], g.rowptr[i + 1]):
            W[i, g.colidx[e]] = g.val[e]
    return W


# --------------------------------------------------------------------------
# §2 / §2.1: W, strengths, L = S - W
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_csr_matches_bruteforce(oracle_mod, seed):
    n, m = 23, 120
    src, dst, w = random_graph(n, m, seed, connected=False)
    # plant explicit duplicates with different weights and self-loops
    src = np.concatenate([src, [3, 5, 7, 7]]).astype(np.int32)
    dst = np.concatenate([dst, [4, 3, 7, 7]]).astype(np.int32)
    w = np.concatenate([w, [9.0, 0.01, 1.0, 2.0]])
    g = oracle_mod.csr_build(n, src, dst, w)
    W = dense_w(n, src, dst, w)
    np.testing.assert_array_equal(to_dense(g), W)
    # columns strictly increasing within rows, no diagonal
    for i in range(n):
        cols = g.colidx[g.rowptr[i]:g.rowptr[i + 1]]
        assert np.all(np.diff(cols) > 0)
        assert i not in cols
    assert g.nnz == int((W > 0).sum())  # all planted weights are positive


def test_csr_empty_and_isolated(oracle_mod):
    g = oracle_mod.csr_build(5, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0))
    assert g.nnz == 0 and list(g.rowptr) == [0] * 6
    g = oracle_mod.csr_build(6, [0, 0], [0, 5], [1.0, 2.0])
    assert list(g.rowptr) == [0, 1, 1, 1, 1, 1, 2]
    assert list(g.colidx) == [5, 0]


def test_csr_rejects_bad_input(oracle_mod):
    with pytest.raises(ValueError):
        oracle_mod.csr_build(3, [0], [3], [1.0])
    with pytest.raises(ValueError):
        oracle_mod.csr_build(3, [0], [1], [-1.0])
    with pytest.raises(ValueError):
        oracle_mod.csr_build(3, [0], [1], [float("nan")])


def test_strength_and_laplacian_null_vector(oracle_mod):
    src, dst, w = random_graph(40, 200, 7)
    g = oracle_mod.csr_build(40, src, dst, w)
    s = oracle_mod.strength(g)
    W = dense_w(40, src, dst, w)
    np.testing.assert_allclose(s, W.sum(axis=1), rtol=1e-14)
    assert math.isclose(s.sum(), g.val.sum(), rel_tol=1e-13)
    L = dense_laplacian(W)
    np.testing.assert_allclose(L @ np.ones(40), 0.0, atol=1e-12)


# --------------------------------------------------------------------------
# §4.1 step 1: lambda_N
# --------------------------------------------------------------------------

def _named_graph(kind, n):
    if kind == "path":
        return np.arange(n - 1), np.arange(1, n)
    if kind == "cycle":
        return np.arange(n), (np.arange(n) + 1) % n
    if kind == "complete":
        i, j = np.triu_indices(n, 1)
        return i, j
    if kind == "star":
        return np.zeros(n - 1, int), np.arange(1, n)
    raise ValueError(kind)


def test_lanczos_closed_form_spectra(oracle_mod):
    rows = []
    with open(os.path.join(GOLDEN, "closed_form_spectra.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                kind, n, lam = line.split()
                rows.append((kind, int(n), float(lam)))
    assert len(rows) >= 8
    rng = np.random.default_rng(3)
    for kind, n, lam in rows:
        src, dst = _named_graph(kind, n)
        g = oracle_mod.csr_build(n, src, dst)
        th = oracle_mod.lanczos_max(g, n, rng.standard_normal(n))
        assert abs(th - lam) <= 1e-10 * lam, (kind, n, th, lam)


def test_lanczos_random_graph_vs_dense(oracle_mod):
    n = 150
    src, dst, w = random_graph(n, 900, 11)
    g = oracle_mod.csr_build(n, src, dst, w)
    ev = np.linalg.eigvalsh(dense_laplacian(dense_w(n, src, dst, w)))
    th = oracle_mod.lanczos_max(g, 80, np.random.default_rng(0).standard_normal(n))
    assert abs(th - ev[-1]) <= 1e-9 * ev[-1]
    # Ritz values never exceed the spectrum; lambda_hat brackets lambda_N
    th5 = oracle_mod.lanczos_max(g, 5, np.random.default_rng(0).standard_normal(n))
    assert th5 <= ev[-1] * (1 + 1e-12)
    lh = oracle_mod.lambda_hat(th, oracle_mod.strength(g))
    assert ev[-1] <= lh <= 2 * oracle_mod.strength(g).max() + 1e-12


def test_tridiag_max_eig_vs_dense():
    import oracle as O
    rng = np.random.default_rng(5)
    for k in (1, 2, 7, 30):
        a = rng.standard_normal(k)
        b = rng.standard_normal(max(k - 1, 0))
        T = np.diag(a) + np.diag(b, 1) + np.diag(b, -1)
        assert abs(O.tridiag_max_eig(a, b) - np.linalg.eigvalsh(T)[-1]) < 1e-12 * (1 + abs(a).max())


# --------------------------------------------------------------------------
# Coefficients of the ideal low-pass (2) in the Chebyshev basis
# --------------------------------------------------------------------------

@pytest.mark.parametrize("frac", [0.013, 0.2, 0.5, 0.77])
def test_coeffs_match_projection_quadrature(oracle_mod, frac):
    lam_max, p = 7.3, 25
    lc = frac * lam_max
    a = oracle_mod.cheb_coeffs(lam_max, lc, p, jackson=False)[0]
    xc = 2 * lc / lam_max - 1
    for j in range(p + 1):
        # (2/pi) int_{-1}^{xc} T_j(x) (1-x)^(-1/2) (1+x)^(-1/2) dx; quad's
        # algebraic weight handles the (1+x)^(-1/2) end point singularity
        tj = np.polynomial.chebyshev.Chebyshev.basis(j)
        val, _ = integrate.quad(lambda x: tj(x) / math.sqrt(1.0 - x), -1.0, xc, weight="alg",
                                wvar=(-0.5, 0.0), limit=400, epsabs=1e-13, epsrel=1e-12)
        ref = (2 / np.pi) * val * (0.5 if j == 0 else 1.0)
        assert abs(a[j] - ref) < 1e-10, (j, a[j], ref)


def test_coeffs_special_cases(oracle_mod):
    p = 12
    a = oracle_mod.cheb_coeffs(3.0, 3.0, p, jackson=True)[0]
    np.testing.assert_allclose(a, np.eye(p + 1)[0], atol=1e-15)
    a = oracle_mod.cheb_coeffs(3.0, 0.0, p, jackson=False)[0]
    np.testing.assert_allclose(a, 0.0, atol=1e-15)
    # cutoff at the middle: the step is odd about x = 0 plus 1/2, so even
    # coefficients beyond a_0 vanish and a_0 = 1/2
    a = oracle_mod.cheb_coeffs(3.0, 1.5, p, jackson=False)[0]
    assert abs(a[0] - 0.5) < 1e-15
    np.testing.assert_allclose(a[2::2], 0.0, atol=1e-15)
    # h_lc(lambda) = 1 for lambda <= lc: at lambda = 0 (x = -1) the undamped
    # series converges to 1 away from the cutoff
    a = oracle_mod.cheb_coeffs(1.0, 0.6, 4000, jackson=False)[0]
    assert abs(cheb_eval(a, -1.0) - 1.0) < 2e-3
    assert abs(cheb_eval(a, 1.0)) < 2e-3


def test_jackson_factors(oracle_mod):
    for p in (1, 5, 50, 200):
        g = oracle_mod.jackson(p)
        assert abs(g[0] - 1.0) < 1e-14
        assert abs(g[1] - math.cos(math.pi / (p + 2))) < 1e-14
        assert np.all(np.diff(g) < 0) and g[-1] > 0


@pytest.mark.parametrize("p", [10, 50, 200])
def test_jackson_damped_step_stays_in_unit_interval(oracle_mod, p):
    """The Jackson kernel is non-negative, so a damped [0, 1]-valued step
    stays in [0, 1]; the undamped series overshoots (Gibbs)."""
    x = np.linspace(-1, 1, 4001)
    for lc in (0.05, 0.3, 0.61):
        yd = cheb_eval(oracle_mod.cheb_coeffs(1.0, lc, p, True)[0], x)
        assert yd.min() > -1e-12 and yd.max() < 1 + 1e-12
        yu = cheb_eval(oracle_mod.cheb_coeffs(1.0, lc, p, False)[0], x)
        assert yu.max() > 1.02


# --------------------------------------------------------------------------
# Fast filtering (3)/(6)/(11) against the exact spectral definition
# --------------------------------------------------------------------------

@pytest.mark.parametrize("jackson", [True, False])
def test_filter_equals_dense_spectral_polynomial(oracle_mod, jackson):
    n, n_sig, p = 70, 5, 33
    src, dst, w = random_graph(n, 300, 21)
    g = oracle_mod.csr_build(n, src, dst, w)
    L = dense_laplacian(dense_w(n, src, dst, w))
    lam, chi = np.linalg.eigh(L)
    lam_max = 1.01 * lam[-1]
    R = np.random.default_rng(1).standard_normal((n, n_sig))
    cut = [0.1 * lam_max, 0.45 * lam_max]
    a = oracle_mod.cheb_coeffs(lam_max, cut, p, jackson)
    Y = oracle_mod.cheb_filter(g, lam_max, a, R)
    lt = 2 * lam / lam_max - 1
    for q in range(2):
        ref = chi @ (cheb_eval(a[q], lt)[:, None] * (chi.T @ R))
        err = np.linalg.norm(Y[q] - ref) / np.linalg.norm(ref)
        assert err < 1e-11, err


def test_filter_p1_and_p2_closed_form(oracle_mod):
    n = 30
    src, dst, w = random_graph(n, 80, 4)
    g = oracle_mod.csr_build(n, src, dst, w)
    L = dense_laplacian(dense_w(n, src, dst, w))
    lam_max = 2.0 * np.abs(L).sum(axis=1).max()
    Lt = 2 * L / lam_max - np.eye(n)
    R = np.random.default_rng(2).standard_normal((n, 3))
    a = np.array([[0.3, -0.7, 0.25]])
    Y = oracle_mod.cheb_filter(g, lam_max, a, R)[0]
    ref = 0.3 * R - 0.7 * Lt @ R + 0.25 * (2 * Lt @ Lt @ R - R)
    np.testing.assert_allclose(Y, ref, rtol=1e-12, atol=1e-12)


def test_projector_identity_and_truncation_error_shrinks(oracle_mod):
    """(5): H_lk = U U^T; the polynomial filter approaches it as p grows
    (measured outside a band around the cutoff, where the step is smooth)."""
    k, m = 4, 30
    n = k * m
    rng = np.random.default_rng(8)
    src, dst = [], []
    for c in range(k):
        for i in range(m):
            for j in range(i + 1, m):
                if rng.random() < 0.3:
                    src.append(c * m + i); dst.append(c * m + j)
    for _ in range(12):
        a_, b_ = rng.integers(0, n, 2)
        src.append(a_); dst.append(b_)
    src, dst = np.array(src, np.int32), np.array(dst, np.int32)
    W = dense_w(n, src, dst)
    lam, chi = np.linalg.eigh(dense_laplacian(W))
    U = chi[:, :k]
    lc = 0.5 * (lam[k - 1] + lam[k])
    H = chi @ np.diag((lam <= lc).astype(float)) @ chi.T
    np.testing.assert_allclose(H, U @ U.T, atol=1e-10)
    g = oracle_mod.csr_build(n, src, dst)
    lam_max = 1.01 * lam[-1]
    R = rng.standard_normal((n, 6))
    band = 0.03 * lam_max
    far = np.abs(lam - lc) > band
    errs = []
    for p in (10, 20, 40, 80, 160):
        Y = oracle_mod.cheb_filter(g, lam_max, oracle_mod.cheb_coeffs(lam_max, lc, p, True), R)[0]
        E = chi.T @ (Y - H @ R)
        errs.append(np.linalg.norm(E[far]) / np.linalg.norm((chi.T @ (H @ R))[far] + 1e-300))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 0.05, errs


def test_disconnected_components_give_constant_features(oracle_mod):
    """§2.1: lambda_1 = 0 has one eigenvector per component (the indicator);
    with lc below every component's lambda_2 the ideal filter is block-constant,
    so normalised features are equal within each component."""
    rng = np.random.default_rng(12)
    sizes = [15, 22, 30]
    src, dst, base = [], [], 0
    for s in sizes:
        for i in range(s):
            for j in range(i + 1, s):
                if rng.random() < 0.6:
                    src.append(base + i); dst.append(base + j)
        base += s
    n = base
    src, dst = np.array(src, np.int32), np.array(dst, np.int32)
    W = dense_w(n, src, dst)
    lam = np.linalg.eigvalsh(dense_laplacian(W))
    assert np.sum(lam < 1e-9) == len(sizes)
    lam2 = lam[len(sizes)]
    lam_max = 1.01 * lam[-1]
    g = oracle_mod.csr_build(n, src, dst)
    a = oracle_mod.cheb_coeffs(lam_max, 0.5 * lam2, 300, True)
    R = np.random.default_rng(3).standard_normal((n, 8)) / np.sqrt(8)
    F = oracle_mod.features(oracle_mod.cheb_filter(g, lam_max, a, R)[0], True)
    base = 0
    for s in sizes:
        blk = F[base:base + s]
        assert np.abs(blk - blk.mean(axis=0)).max() < 2e-3
        base += s


# --------------------------------------------------------------------------
# §3.2 eigenvalue count and dichotomy
# --------------------------------------------------------------------------

def test_eigencount_matches_expectation(oracle_mod):
    n, eta, p = 120, 64, 60
    src, dst, w = random_graph(n, 500, 31)
    g = oracle_mod.csr_build(n, src, dst, w)
    lam = np.linalg.eigvalsh(dense_laplacian(dense_w(n, src, dst, w)))
    lam_max = 1.01 * lam[-1]
    R = np.random.default_rng(4).standard_normal((n, eta)) / np.sqrt(eta)
    cut = np.array([0.05, 0.2, 0.5]) * lam_max
    a = oracle_mod.cheb_coeffs(lam_max, cut, p, True)
    cnt = oracle_mod.eigencount(g, lam_max, a, R)
    lt = 2 * lam / lam_max - 1
    for q in range(3):
        P = cheb_eval(a[q], lt)
        mean = np.sum(P ** 2)
        sd = math.sqrt(2 * np.sum(P ** 4) / eta)
        assert abs(cnt[q] - mean) < 4 * sd, (q, cnt[q], mean, sd)
        # and the count tracks the number of eigenvalues below the cutoff
        assert abs(mean - np.sum(lam <= cut[q])) < 0.15 * n


def test_moments_vs_dense_and_direct_count(oracle_mod):
    n, eta, p = 60, 7, 20
    src, dst, w = random_graph(n, 240, 41)
    g = oracle_mod.csr_build(n, src, dst, w)
    lam, chi = np.linalg.eigh(dense_laplacian(dense_w(n, src, dst, w)))
    lam_max = 1.01 * lam[-1]
    R = np.random.default_rng(5).standard_normal((n, eta))
    mu = oracle_mod.moments(g, lam_max, R, 2 * p)
    lt = 2 * lam / lam_max - 1
    Rh2 = np.sum((chi.T @ R) ** 2, axis=1)
    for m in range(2 * p + 1):
        ref = np.sum(Rh2 * np.cos(m * np.arccos(np.clip(lt, -1, 1))))
        assert abs(mu[m] - ref) < 1e-10 * np.sum(Rh2)
    a = oracle_mod.cheb_coeffs(lam_max, [0.1 * lam_max, 0.3 * lam_max], p, True)
    direct = oracle_mod.eigencount(g, lam_max, a, R)
    via = oracle_mod.count_from_moments(mu, a)
    np.testing.assert_allclose(via, direct, rtol=1e-10)


def test_dichotomy_on_disjoint_cliques(oracle_mod):
    """k disjoint K_m: eigenvalues 0 (k times) and m. The dichotomy finds a
    cutoff inside [0, m) whose count reaches k, and just below it the count
    is below k."""
    k, m, eta, p = 5, 8, 200, 80
    src, dst = cliques_edges(k, m)
    n = k * m
    g = oracle_mod.csr_build(n, src, dst)
    lam_max = 1.01 * m
    R = np.random.default_rng(6).standard_normal((n, eta)) / np.sqrt(eta)
    lk = oracle_mod.dichotomy(g, lam_max, p, R, k - 0.5, True, 40, 1e-9)
    assert 0.0 < lk < m
    a_hi = oracle_mod.cheb_coeffs(lam_max, lk, p, True)
    a_lo = oracle_mod.cheb_coeffs(lam_max, lk - 2e-9 * lam_max, p, True)
    assert oracle_mod.eigencount(g, lam_max, a_hi, R)[0] >= k - 0.5
    assert oracle_mod.eigencount(g, lam_max, a_lo, R)[0] < k - 0.5


def test_dichotomy_matches_spectral_bisection(oracle_mod):
    """With the identity as the signal block the count is exact,
    ||F I||_F^2 = tr(P(Lt)^2) = sum_l P(lt_l)^2, so the dichotomy must land on
    the cutoff an independent bisection finds from the dense spectrum (numpy's
    eigensolver and Chebyshev evaluation), for targets between and on the
    plateaus of the count."""
    n = 48
    src, dst, w = random_graph(n, 260, 5)
    g = oracle_mod.csr_build(n, src, dst, w)
    lam = np.linalg.eigvalsh(dense_laplacian(dense_w(n, src, dst, w)))
    lam_max = 1.01 * lam[-1]
    p = 40
    R = np.eye(n)

    def count(lc):
        a = oracle_mod.cheb_coeffs(lam_max, lc, p, True)[0]
        return float(np.sum(cheb_eval(a, 2 * lam / lam_max - 1) ** 2))

    for target in (2.5, 7.2, 15.5, 30.0):
        lo, hi = 0.0, lam_max
        for _ in range(40):
            if hi - lo <= 1e-9 * lam_max:
                break
            mid = 0.5 * (lo + hi)
            if count(mid) >= target:
                hi = mid
            else:
                lo = mid
        got = oracle_mod.dichotomy(g, lam_max, p, R, target, True, 40, 1e-9)
        assert got == pytest.approx(hi, rel=1e-12, abs=1e-12)


# --------------------------------------------------------------------------
# Features (6)/(11)
# --------------------------------------------------------------------------

def test_features(oracle_mod):
    rng = np.random.default_rng(9)
    Y = rng.standard_normal((50, 9))
    Y[7] = 0.0
    F = oracle_mod.features(Y, True)
    nr = np.linalg.norm(F, axis=1)
    np.testing.assert_allclose(np.delete(nr, 7), 1.0, rtol=1e-14)
    assert np.all(F[7] == 0.0)
    np.testing.assert_allclose(F * np.linalg.norm(Y, axis=1, keepdims=True), Y, rtol=1e-14, atol=1e-15)
    np.testing.assert_array_equal(oracle_mod.features(Y, False), Y)


def test_jl_proposition_distances(oracle_mod):
    """Proposition of §3.1: with eta >= eta_0, all pairwise feature distances
    are preserved within (1 +- eps) with probability >= 1 - N^-beta
    (exact filter H_lk = U U^T on a small graph, fixed seed)."""
    n, k = 40, 4
    src, dst = cliques_edges(k, n // k)
    rng = np.random.default_rng(14)
    src = np.concatenate([src, rng.integers(0, n, 6)]).astype(np.int32)
    dst = np.concatenate([dst, rng.integers(0, n, 6)]).astype(np.int32)
    lam, chi = np.linalg.eigh(dense_laplacian(dense_w(n, src, dst)))
    U = chi[:, :k]
    eps, beta = 0.5, 1.0
    eta0 = (4 + 2 * beta) / (eps ** 2 / 2 - eps ** 3 / 3) * math.log(n)
    eta = int(math.ceil(eta0))
    R = rng.standard_normal((n, eta)) / math.sqrt(eta)
    Ft = (U @ U.T) @ R
    f = U
    i, j = np.triu_indices(n, 1)
    d = np.sum((f[i] - f[j]) ** 2, axis=1)
    dt = np.sum((Ft[i] - Ft[j]) ** 2, axis=1)
    mask = d > 1e-12
    ratio = dt[mask] / d[mask]
    assert ratio.min() >= 1 - eps and ratio.max() <= 1 + eps


# --------------------------------------------------------------------------
# Reverse mode (adjoint) against central finite differences
# --------------------------------------------------------------------------

def test_backward_matches_finite_differences(oracle_mod):
    n, n_sig, p = 14, 3, 7
    src, dst, w = random_graph(n, 30, 51)
    g = oracle_mod.csr_build(n, src, dst, w)
    s = oracle_mod.strength(g)
    lam_max = 2.0 * s.max()
    rng = np.random.default_rng(7)
    R = rng.standard_normal((n, n_sig))
    G = rng.standard_normal((n, n_sig))
    a = oracle_mod.cheb_coeffs(lam_max, 0.3 * lam_max, p, True)[0]
    gv, ga, gR = oracle_mod.cheb_filter_backward(g, lam_max, a, R, G, want_grad_R=True)

    def loss(val=None, a_=None, R_=None):
        gg = oracle_mod.CSR(g.n, g.rowptr, g.colidx, g.val if val is None else val)
        return float(np.sum(G * oracle_mod.cheb_filter(gg, lam_max, a if a_ is None else a_,
                                                        R if R_ is None else R_)[0]))

    h = 1e-6
    # each undirected edge: perturb both stored directions together
    checked = 0
    for u in range(n):
        for e in range(g.rowptr[u], g.rowptr[u + 1]):
            v = g.colidx[e]
            if v < u:
                continue
            f = [ff for ff in range(g.rowptr[v], g.rowptr[v + 1]) if g.colidx[ff] == u][0]
            vp, vm = g.val.copy(), g.val.copy()
            vp[e] += h; vp[f] += h; vm[e] -= h; vm[f] -= h
            fd = (loss(val=vp) - loss(val=vm)) / (2 * h)
            assert abs(fd - gv[e]) <= 1e-6 * max(1.0, abs(fd)), (u, v, fd, gv[e])
            assert abs(gv[e] - gv[f]) <= 1e-13 * max(1.0, abs(gv[e]))
            checked += 1
    assert checked > 10
    for j in range(p + 1):
        ap, am = a.copy(), a.copy()
        ap[j] += h; am[j] -= h
        fd = (loss(a_=ap) - loss(a_=am)) / (2 * h)
        assert abs(fd - ga[j]) <= 1e-6 * max(1.0, abs(fd))
    for (i, r) in [(0, 0), (5, 2), (13, 1)]:
        Rp, Rm = R.copy(), R.copy()
        Rp[i, r] += h; Rm[i, r] -= h
        fd = (loss(R_=Rp) - loss(R_=Rm)) / (2 * h)
        assert abs(fd - gR[i, r]) <= 1e-6 * max(1.0, abs(fd))


# ------------------------------------------------------------------ k-means (§4.1 step 6)
def test_kmeans_assignment_is_bruteforce_argmin_and_update_is_mean(oracle_mod):
    """One Lloyd iteration: labels equal numpy's FP64 argmin of squared
    distances wherever the best two candidates are not within FP32 rounding,
    and the new centroids are the numpy means of the labelled rows."""
    rng = np.random.default_rng(3)
    n, d, k = 2000, 24, 9
    F = rng.standard_normal((n, d)).astype(np.float32)
    C0 = rng.standard_normal((k, d)).astype(np.float32)
    labels, C1, iters, inertia = oracle_mod.kmeans(F, C0, 1)
    assert iters == 1
    D = ((F.astype(np.float64)[:, None, :] - C0.astype(np.float64)[None, :, :]) ** 2).sum(-1)
    srt = np.sort(D, axis=1)
    clear = (srt[:, 1] - srt[:, 0]) > 1e-4 * srt[:, 1]
    assert clear.mean() > 0.99
    np.testing.assert_array_equal(labels[clear], np.argmin(D, axis=1)[clear])
    assert inertia == pytest.approx(D[np.arange(n), labels].sum(), rel=1e-5)
    for c in range(k):
        rows = F[labels == c].astype(np.float64)
        if len(rows):
            np.testing.assert_allclose(C1[c], rows.mean(axis=0), rtol=1e-6, atol=1e-7)
        else:
            np.testing.assert_array_equal(C1[c], C0[c])


def test_kmeans_recovers_separated_clusters(oracle_mod):
    """Points scattered tightly around k far-apart centres, started from one
    point of each cluster: labels equal the generating clusters and centroids
    their means after two assignments (the second changes nothing)."""
    rng = np.random.default_rng(4)
    k, d, per = 6, 5, 150
    centres = rng.standard_normal((k, d)) * 50.0
    truth = np.repeat(np.arange(k), per)
    F = (centres[truth] + rng.standard_normal((k * per, d)) * 0.5).astype(np.float32)
    C0 = F[np.arange(k) * per].copy()
    labels, C, iters, _ = oracle_mod.kmeans(F, C0, 20)
    np.testing.assert_array_equal(labels, truth)
    assert iters == 2
    for c in range(k):
        np.testing.assert_allclose(C[c], F[truth == c].astype(np.float64).mean(axis=0), rtol=1e-6, atol=1e-6)


def test_kmeans_inertia_never_increases(oracle_mod):
    """Lloyd's iterations never increase the inertia (each step minimises it
    over labels, then over centroids)."""
    rng = np.random.default_rng(5)
    F = rng.standard_normal((1500, 8)).astype(np.float32)
    C0 = F[rng.choice(1500, 12, replace=False)].copy()
    prev = math.inf
    for t in range(1, 12):
        _, _, iters, inertia = oracle_mod.kmeans(F, C0, t)
        assert inertia <= prev * (1 + 1e-9)
        prev = inertia
        if iters < t:
            break


def test_kmeans_ties_and_empty_clusters(oracle_mod):
    """Equal centroids: every row takes the lower index. A centroid no row is
    nearest to keeps its coordinates."""
    rng = np.random.default_rng(6)
    F = rng.standard_normal((300, 4)).astype(np.float32)
    C0 = np.stack([np.zeros(4), np.zeros(4), np.full(4, 1e6)]).astype(np.float32)
    labels, C, iters, _ = oracle_mod.kmeans(F, C0, 1)
    assert np.all(labels == 0)
    np.testing.assert_array_equal(C[1], C0[1])
    np.testing.assert_array_equal(C[2], C0[2])


# ------------------------------------------------------------------ normalised Laplacian (footnote of §2.1)
def _dense_from_csr(g):
    """Dense L = diag(d) - W' of an oracle CSR (with its explicit diagonal when set)."""
    n = g.n
    W = np.zeros((n, n))
    for i in range(n):
        for e in range(g.rowptr[i], g.rowptr[i + 1]):
            W[i, g.colidx[e]] = g.val[e]
    d = W.sum(1) if g.diag is None else np.asarray(g.diag)
    return np.diag(d) - W


def test_normalized_laplacian_closed_form_spectra(oracle_mod):
    """K_n: eigenvalues 0 and n/(n-1) (n-1 times); C_n (2-regular): 1 - cos(2 pi j / n);
    a connected bipartite graph (star S_n) has eigenvalues 0, 1 (n-2 times) and 2."""
    n = 9
    s, d = np.triu_indices(n, 1)
    ev = np.linalg.eigvalsh(_dense_from_csr(oracle_mod.normalize(oracle_mod.csr_build(n, s, d))))
    np.testing.assert_allclose(ev, np.r_[0.0, np.full(n - 1, n / (n - 1))], atol=1e-12)
    n = 11
    s = np.arange(n)
    ev = np.linalg.eigvalsh(_dense_from_csr(oracle_mod.normalize(oracle_mod.csr_build(n, s, (s + 1) % n))))
    np.testing.assert_allclose(ev, np.sort(1 - np.cos(2 * np.pi * np.arange(n) / n)), atol=1e-12)
    n = 7
    ev = np.linalg.eigvalsh(_dense_from_csr(oracle_mod.normalize(oracle_mod.csr_build(n, np.zeros(n - 1, int),
                                                                                        np.arange(1, n)))))
    np.testing.assert_allclose(ev, np.r_[0.0, np.ones(n - 2), 2.0], atol=1e-12)


def test_normalized_laplacian_matches_dense_definition(oracle_mod):
    """Against I - S^{-1/2} W S^{-1/2} built densely from the edge list, with
    an isolated node (its row and column stay 0): same matrix, null vector
    S^{1/2} 1 on the connected part, spectrum inside [0, 2]."""
    n = 60
    src, dst, w = random_graph(n - 1, 400, 13)  # node n - 1 isolated
    g = oracle_mod.csr_build(n, src, dst, w)
    Ln = _dense_from_csr(oracle_mod.normalize(g))
    W = dense_w(n, src, dst, w)
    s = W.sum(1)
    dinv = np.where(s > 0, 1.0 / np.sqrt(np.where(s > 0, s, 1.0)), 0.0)
    ref = np.diag((s > 0).astype(float)) - dinv[:, None] * W * dinv[None, :]
    np.testing.assert_allclose(Ln, ref, atol=1e-14)
    np.testing.assert_allclose(Ln @ np.sqrt(s), 0.0, atol=1e-12)
    ev = np.linalg.eigvalsh(Ln)
    assert ev.min() > -1e-12 and ev.max() < 2 + 1e-12


def test_filter_on_normalized_laplacian_equals_spectral_polynomial(oracle_mod):
    """The explicit-diagonal filter equals chi P(Lt) chi^T R for the dense
    normalised Laplacian (lam_hat = 2, its spectral bound)."""
    n, p = 80, 30
    src, dst, w = random_graph(n, 500, 17)
    gn = oracle_mod.normalize(oracle_mod.csr_build(n, src, dst, w))
    lam, chi = np.linalg.eigh(_dense_from_csr(gn))
    lh = 2.0
    a = oracle_mod.cheb_coeffs(lh, 0.4, p, True)[0]
    R = np.random.default_rng(3).standard_normal((n, 5))
    Y = oracle_mod.cheb_filter(gn, lh, a, R)[0]
    ref = chi @ (cheb_eval(a, 2 * lam / lh - 1)[:, None] * (chi.T @ R))
    np.testing.assert_allclose(Y, ref, atol=1e-11)


# ------------------------------------------------------------------ stability (§4.3, Eq. (12))
def _ari_bruteforce(a, b):
    """Adjusted Rand index by counting every pair of items (Hubert and Arabie):
    pairs together in both, in a only, in b only."""
    n = len(a)
    both = in_a = in_b = 0
    for i in range(n):
        for j in range(i + 1, n):
            sa, sb = a[i] == a[j], b[i] == b[j]
            both += sa and sb
            in_a += sa
            in_b += sb
    pairs = n * (n - 1) / 2
    expected = in_a * in_b / pairs
    top = 0.5 * (in_a + in_b)
    return 1.0 if top == expected else (both - expected) / (top - expected)


def test_adjusted_rand_index(oracle_mod):
    rng = np.random.default_rng(9)
    for n, ka, kb in ((40, 3, 4), (57, 5, 2), (25, 1, 3)):
        a = rng.integers(0, ka, n)
        b = rng.integers(0, kb, n)
        assert oracle_mod.adjusted_rand(a, b) == pytest.approx(_ari_bruteforce(a, b), abs=1e-12)
    a = rng.integers(0, 6, 500)
    assert oracle_mod.adjusted_rand(a, a) == 1.0
    assert oracle_mod.adjusted_rand(a, (a * 5 + 1) % 6) == pytest.approx(1.0)  # relabelled
    assert abs(oracle_mod.adjusted_rand(a, rng.integers(0, 6, 500))) < 0.05


def test_stability_peaks_at_the_true_number_of_clusters(oracle_mod):
    """Eq. (12) on k well-separated communities (dense blocks, few links
    between them), k-means with 8 seeded starts per clustering: every
    realisation finds the same partition at the true k (gamma = 1), and the
    other candidates are less stable."""
    k, m = 4, 40
    n = k * m
    rng = np.random.default_rng(21)
    src, dst = [], []
    for c in range(k):
        for i in range(m):
            for j in range(i + 1, m):
                if rng.random() < 0.5:
                    src.append(c * m + i)
                    dst.append(c * m + j)
    for _ in range(12):  # sparse links between communities
        u, v = rng.integers(0, n, 2)
        src.append(u)
        dst.append(v)
    g = oracle_mod.csr_build(n, np.array(src), np.array(dst))
    s = oracle_mod.strength(g)
    th = oracle_mod.lanczos_max(g, 60, rng.standard_normal(n))
    lh = oracle_mod.lambda_hat(th, s)
    eta = 12
    Rc = rng.standard_normal((n, eta)) / np.sqrt(eta)
    Rs = [rng.standard_normal((n, eta)) / np.sqrt(eta) for _ in range(4)]
    gamma, lam_k = oracle_mod.stability(g, lh, 60, Rc, Rs, 2, 6, 50, 7, starts=8)
    assert gamma[k - 2] == pytest.approx(1.0)
    assert np.argmax(gamma) == k - 2
    assert np.all(np.diff(lam_k) >= 0)  # more clusters, higher cutoff
    # sharper filters (order 3p) at the same count cutoffs: the same cutoffs; the clusterings stay
    # identical up to the true k and become unstable beyond it
    gamma3, lam_k3 = oracle_mod.stability(g, lh, 60, Rc, Rs, 2, 6, 50, 7, starts=8, p_filter=180)
    np.testing.assert_array_equal(lam_k3, lam_k)
    assert gamma3[k - 2] == pytest.approx(1.0) and np.all(gamma3[k - 1:] < 1.0 - 1e-3)
    # the init rule is SplitMix64 (Steele, Lea and Flood 2014) of the packed counter, mod n
    z = (7 + (((1 << 40) | (3 << 20) | (5 << 10) | 2) + 1) * 0x9E3779B97F4A7C15) & (2**64 - 1)
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & (2**64 - 1)
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & (2**64 - 1)
    z ^= z >> 31
    assert oracle_mod.stability_init_row(7, 1, 3, 5, 2, n) == z % n


# ------------------------------------------------------------------ order table m* (§2.4, criterion (4))
def test_cheb_order_matches_chebval_search(oracle_mod):
    """m* against a search with numpy's Chebyshev evaluation (library routine)
    on the same points, and its monotonicity: a looser tolerance or a wider
    excluded band never needs a higher order."""
    def search(x, delta, w, jackson, p_max=400):
        t = np.r_[np.arange(4096) / 4095.0, [x - w] if x - w >= 0 else [], [x + w] if x + w <= 1 else []]
        t = t[np.abs(t - x) >= w]
        h = (t <= x).astype(float)
        for m in range(1, p_max + 1):
            a = oracle_mod.cheb_coeffs(1.0, x, m, jackson)[0]
            if np.max(np.abs(h - cheb_eval(a, 2 * t - 1))) <= delta:
                return m
        return -1

    for x, delta, w, jk in ((0.3, 0.1, 0.05, True), (0.1, 0.1, 0.02, True), (0.7, 0.05, 0.1, True),
                            (0.5, 0.2, 0.1, False)):
        assert oracle_mod.cheb_order(x, delta, w, jk, 400) == search(x, delta, w, jk)
    base = oracle_mod.cheb_order(0.2, 0.1, 0.03)
    assert oracle_mod.cheb_order(0.2, 0.2, 0.03) <= base
    assert oracle_mod.cheb_order(0.2, 0.1, 0.06) <= base
    # the undamped series overshoots by ~9% just outside the jump (Gibbs): with a band too narrow to hide the
    # first overshoot, delta = 0.05 is out of reach; the damped series (a positive kernel) never overshoots
    assert oracle_mod.cheb_order(0.4, 0.05, 1e-4, False, 300) == -1
    assert oracle_mod.cheb_order(0.4, 0.05, 0.01, True, 2000) > 0


def test_parallel_build_equals_plain_build(oracle_mod):
    """The OpenMP build of the oracle (the timed CPU baseline on all host cores)
    computes every element with the same operations in the same order as the
    plain build: identical filter outputs, for any number of threads."""
    from helpers import random_graph

    oracle_mod.build_parallel()
    n = 700
    src, dst, w = random_graph(n, 6000, seed=21)
    g = oracle_mod.csr_build(n, src, dst, w)
    lam = 2.0 * float(oracle_mod.strength(g).max())
    a = oracle_mod.cheb_coeffs(lam, [0.1 * lam, 0.3 * lam], 17, True)
    R = np.random.default_rng(3).standard_normal((n, 5))
    Y1 = oracle_mod.cheb_filter(g, lam, a, R)
    Yp = oracle_mod.cheb_filter(g, lam, a, R, parallel=True)
    assert oracle_mod.threads() == 1
    assert oracle_mod.threads(parallel=True) >= 1
    np.testing.assert_array_equal(Y1, Yp)
