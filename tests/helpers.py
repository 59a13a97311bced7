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
