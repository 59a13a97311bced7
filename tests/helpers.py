"""Small, independent helpers for the pins: dense matrices built straight from
edge lists with Python loops (never from either implementation's CSR)."""
import numpy as np


def dense_w(n, src, dst, w=None):
    """Dense symmetric W: self-loops dropped, repeated pairs merged by max."""
    W = np.zeros((n, n))
    if w is None:
        w = np.ones(len(src))
    for u, v, x in zip(src, dst, w):
        u, v = int(u), int(v)
        if u == v:
            continue
        W[u, v] = max(W[u, v], float(x))
        W[v, u] = max(W[v, u], float(x))
    return W


def dense_laplacian(W):
    return np.diag(W.sum(axis=1)) - W


def random_graph(n, m, seed, weighted=True, connected=True):
    """Random multigraph edge list (with repeats and self-loops); a spanning
    path is added when `connected`."""
    rng = np.random.default_rng(seed)
    src = rng.integers(0, n, m)
    dst = rng.integers(0, n, m)
    if connected:
        perm = rng.permutation(n)
        src = np.concatenate([src, perm[:-1]])
        dst = np.concatenate([dst, perm[1:]])
    w = rng.uniform(0.1, 2.0, len(src)) if weighted else np.ones(len(src))
    return src.astype(np.int32), dst.astype(np.int32), w


def cheb_eval(a, x):
    """sum_j a_j T_j(x) via numpy's Chebyshev module (library routine)."""
    return np.polynomial.chebyshev.chebval(x, a)


def cliques_edges(k, m, seed=0):
    """k disjoint complete graphs K_m (unit weights)."""
    src, dst = [], []
    for c in range(k):
        base = c * m
        for i in range(m):
            for j in range(i + 1, m):
                src.append(base + i)
                dst.append(base + j)
    return np.array(src, np.int32), np.array(dst, np.int32)


def oracle_lambda_hat(oracle_mod, go, iters=60, seed=0):
    """lam_hat for a comparison, computed by the oracle (its Lanczos from a seeded
    start, then the reading of §4.1 step 1); both sides are given this value."""
    v0 = np.random.default_rng(seed).standard_normal(go.n)
    return oracle_mod.lambda_hat(oracle_mod.lanczos_max(go, iters, v0), oracle_mod.strength(go))


def stored_block_error_model(lam_tilde, a, u, algo, input_rounded):
    """Relative Frobenius error of a filter whose blocks are stored with unit
    roundoff u (BF16 2^-8, FP16 2^-11) while sums stay exact, from the spectrum
    lam_tilde of Lt and the coefficients a (length p + 1).

    Model: every stored element is rounded once per order with an error of RMS
    u / sqrt(3) relative to its value, independently across elements and orders,
    so the errors of one order are spread evenly over the spectrum. The error
    injected into T_k (forward recurrence, k >= 1) reaches Y through the tail
    q_k = sum_{j > k} a_j U_{j-k-1}(Lt) (Chebyshev polynomials of the second
    kind: the recurrence's response to a perturbation); with Clenshaw the error
    injected into b_k = sum_{j >= k} a_j U_{j-k}(Lt) reaches Y through
    U_{k-1}(Lt). Rounding the input R itself (input_rounded) adds the filter
    applied to its error. Summing the independent contributions:
        err^2 = (u^2 / 3) [sum_k mean(s_k^2) mean(r_k^2) + input] / mean(P^2),
    with s_k the stored polynomial, r_k its propagator and means over the
    spectrum. It takes every rounding at its largest relative size, so it sits
    above a measured error (by about 2x on the 1000-node SBM)."""
    x = np.asarray(lam_tilde, np.float64)
    a = np.asarray(a, np.float64)
    p = len(a) - 1
    T = np.zeros((p + 2, len(x)))
    U = np.zeros((p + 2, len(x)))
    T[0], T[1], U[0], U[1] = 1.0, x, 1.0, 2.0 * x
    for k in range(2, p + 2):
        T[k] = 2.0 * x * T[k - 1] - T[k - 2]
        U[k] = 2.0 * x * U[k - 1] - U[k - 2]

    def Uk(k):
        return U[k] if k >= 0 else np.zeros_like(x)

    P = a @ T[: p + 1]
    tot = 0.0
    if algo == "forward":
        for k in range(1, p):
            q = sum(a[j] * Uk(j - k - 1) for j in range(k + 1, p + 1))
            tot += np.mean(T[k] ** 2) * np.mean(q ** 2)
    else:
        for k in range(1, p + 1):
            b = sum(a[j] * Uk(j - k) for j in range(k, p + 1))
            tot += np.mean(b ** 2) * np.mean(Uk(k - 1) ** 2)
    tot /= np.mean(P ** 2)
    if input_rounded:
        tot += 1.0
    return u * np.sqrt(tot / 3.0)
