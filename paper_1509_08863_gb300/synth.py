"""Seeded synthetic workloads (graphs, random signal blocks, upstream gradients).

This module only draws inputs. It holds none of the method's arithmetic (no
Laplacian, no filter, no coefficient), so both the CUDA path and the CPU oracle
can be fed from it without sharing any computation.

Workloads follow the shapes of the paper's experiments (§5: similarity graphs
with community structure, kNN graphs on Gaussian-mixture points) at the sizes
the benchmarks and tests use:

* ``sbm_edges``: stochastic block model. Per block pair (a, b) the number of
  candidate edges is Binomial(pairs_ab, p_ab); endpoints are drawn uniformly in
  the two blocks, with replacement. Duplicates and self-loops are therefore
  possible in the edge list; the CSR build removes self-loops and merges
  duplicates (their weights are equal, all 1). Node ids are permuted by a
  seeded permutation so that no memory locality is gifted to the kernels.
  ``p_in = c_in / N`` and ``p_out = eps * p_in`` with ``c_in`` chosen so that
  the expected mean degree equals ``mean_degree``:
  ``p_in * [sum_c n_c (n_c - 1) + eps (N^2 - sum_c n_c^2)] = mean_degree * N``.
* ``knn_mixture_edges``: points from a mixture of Gaussians, directed K-nearest
  neighbour edges with weight exp(-|x_i - x_j|^2 / sigma^2); the CSR build's
  max-merge turns the directed lists into the union graph max(A, A^T).
* ``gaussian_block``: i.i.d. N(0, 1/eta) entries (§3.1: the random signals),
  drawn with the counter-based Philox4x32-10 bit generator of numpy.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "community_sizes_equal",
    "community_sizes_uniform",
    "sbm_edges",
    "knn_mixture_edges",
    "gaussian_block",
    "standard_normal_block",
    "batched_sbm",
    "SBMGraph",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(int(seed)))


def community_sizes_equal(n: int, k: int) -> np.ndarray:
    """k sizes summing to n, differing by at most one."""
    base, rem = divmod(n, k)
    sizes = np.full(k, base, dtype=np.int64)
    sizes[:rem] += 1
    return sizes


def community_sizes_uniform(n: int, k: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """k sizes drawn i.i.d. uniform in [lo, hi], rescaled so that they sum to n.

    The rounding remainder is spread one node at a time over the largest
    communities.
    """
    rng = _rng(seed)
    raw = rng.integers(lo, hi + 1, size=k).astype(np.float64)
    sizes = np.floor(raw * (n / raw.sum())).astype(np.int64)
    sizes = np.maximum(sizes, 1)
    rem = n - int(sizes.sum())
    order = np.argsort(-raw, kind="stable")
    i = 0
    while rem != 0:
        step = 1 if rem > 0 else -1
        j = order[i % k]
        if sizes[j] + step >= 1:
            sizes[j] += step
            rem -= step
        i += 1
    return sizes


class SBMGraph:
    """An edge list with its ground-truth labels."""

    def __init__(self, n, src, dst, w, labels, sizes):
        self.n = int(n)
        self.src = src
        self.dst = dst
        self.w = w
        self.labels = labels
        self.sizes = sizes

    @property
    def n_edges(self) -> int:
        return int(self.src.shape[0])


def sbm_edges(
    n: int,
    sizes: np.ndarray,
    mean_degree: float,
    eps: float,
    seed: int,
    permute: bool = True,
) -> SBMGraph:
    """Stochastic block model edge list (int32 endpoints, float32 unit weights)."""
    sizes = np.asarray(sizes, dtype=np.int64)
    assert int(sizes.sum()) == n
    k = sizes.shape[0]
    rng = _rng(seed)
    sum_sq = float((sizes.astype(np.float64) ** 2).sum())
    denom = float((sizes * (sizes - 1)).sum()) + eps * (float(n) * n - sum_sq)
    p_in = mean_degree * n / denom
    p_out = eps * p_in
    assert p_in <= 1.0, "mean degree too high for the block sizes"
    offs = np.concatenate([[0], np.cumsum(sizes)])

    # Block pairs a <= b and their candidate-pair counts.
    ia, ib = np.triu_indices(k)
    na = sizes[ia].astype(np.float64)
    nb = sizes[ib].astype(np.float64)
    pairs = np.where(ia == ib, na * (na - 1) / 2.0, na * nb)
    prob = np.where(ia == ib, p_in, p_out)
    counts = rng.binomial(pairs.astype(np.int64), prob)
    total = int(counts.sum())
    blk_a = np.repeat(ia, counts)
    blk_b = np.repeat(ib, counts)
    u = offs[blk_a] + np.floor(rng.random(total) * sizes[blk_a]).astype(np.int64)
    v = offs[blk_b] + np.floor(rng.random(total) * sizes[blk_b]).astype(np.int64)
    labels = np.repeat(np.arange(k, dtype=np.int32), sizes)
    if permute:
        perm = rng.permutation(n)  # old id -> new id
        u = perm[u]
        v = perm[v]
        new_labels = np.empty_like(labels)
        new_labels[perm] = labels
        labels = new_labels
    src = u.astype(np.int32)
    dst = v.astype(np.int32)
    w = np.ones(total, dtype=np.float32)
    return SBMGraph(n, src, dst, w, labels, sizes)


def knn_mixture_edges(
    n: int,
    n_comp: int,
    dim: int,
    k_nn: int,
    sigma: float,
    centre_std: float,
    seed: int,
):
    """Directed K-NN edges of points drawn from a Gaussian mixture.

    Components have unit variance and centres drawn N(0, centre_std^2 I); each
    point picks a component uniformly. Returns (src, dst, w float32, labels,
    points). Neighbours are found exactly with a k-d tree; the point itself is
    excluded.
    """
    from scipy.spatial import cKDTree

    rng = _rng(seed)
    centres = rng.standard_normal((n_comp, dim)) * centre_std
    labels = rng.integers(0, n_comp, size=n).astype(np.int32)
    pts = centres[labels] + rng.standard_normal((n, dim))
    tree = cKDTree(pts)
    dist, idx = tree.query(pts, k=k_nn + 1)
    src = np.repeat(np.arange(n, dtype=np.int64), k_nn)
    # Drop the query point itself (first hit unless exact duplicates exist).
    nbr = idx[:, 1:].reshape(-1)
    d2 = dist[:, 1:].reshape(-1) ** 2
    keep = nbr != src
    src, nbr, d2 = src[keep], nbr[keep], d2[keep]
    w = np.exp(-d2 / (sigma * sigma)).astype(np.float32)
    return src.astype(np.int32), nbr.astype(np.int32), w, labels, pts


def standard_normal_block(n: int, cols: int, seed: int) -> np.ndarray:
    """n x cols i.i.d. N(0, 1) float64, row-major."""
    return _rng(seed).standard_normal((n, cols))


def gaussian_block(n: int, eta: int, seed: int) -> np.ndarray:
    """R in R^{n x eta} with i.i.d. N(0, 1/eta) entries, float64 (§3.1, §4.1 step 4)."""
    return standard_normal_block(n, eta, seed) / np.sqrt(eta)


def batched_sbm(n_graphs: int, seed: int, n_lo=1000, n_hi=50000, k_lo=2, k_hi=30,
                d_lo=8.0, d_hi=32.0, eps=0.1):
    """Many independent SBM graphs of uneven size (equal communities per graph).

    Graph g uses seed ``seed + g`` for its edges; its size, community count and
    mean degree are drawn from ``seed`` first.
    """
    rng = _rng(seed)
    ns = rng.integers(n_lo, n_hi + 1, size=n_graphs)
    ks = rng.integers(k_lo, k_hi + 1, size=n_graphs)
    ds = rng.uniform(d_lo, d_hi, size=n_graphs)
    graphs = []
    for g in range(n_graphs):
        sizes = community_sizes_equal(int(ns[g]), int(ks[g]))
        graphs.append(sbm_edges(int(ns[g]), sizes, float(ds[g]), eps, seed + 1 + g))
    return graphs, ks
