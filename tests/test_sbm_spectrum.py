"""Why the method does not recover the communities of the 100k-node SBM with
L = S - W but does with the normalised Laplacian (footnote of §2.1): on the
same recipe at 2,000 nodes (k = 20, sizes uniform in a 1:4 range, mean
degree 20, c_out/c_in = 0.1), a dense eigendecomposition shows the 20 lowest
eigenvectors of L = S - W localised on low-degree nodes, below the community
indicators' Rayleigh quotients, while those of the normalised Laplacian are
spread over the graph and lie largely in the span of the indicators."""
import numpy as np

from paper_1509_08863_gb300 import synth


def _laplacians():
    n, k = 2000, 20
    gr = synth.sbm_edges(n, synth.community_sizes_uniform(n, k, 40, 160, seed=7), 20.0, 0.1, seed=1002)
    W = np.zeros((n, n))
    keep = gr.src != gr.dst
    W[gr.src[keep], gr.dst[keep]] = 1.0
    W = np.maximum(W, W.T)
    s = W.sum(1)
    inv = np.where(s > 0, 1.0 / np.sqrt(np.maximum(s, 1e-300)), 0.0)
    L = np.diag(s) - W
    Ln = np.eye(n) - inv[:, None] * W * inv[None, :]
    Y = np.zeros((n, k))
    Y[np.arange(n), gr.labels] = 1.0
    return L, Ln, Y, s, k


def _stats(M, Y, s, k):
    vals, vecs = np.linalg.eigh(M)
    vals, vecs = vals[:k], vecs[:, :k]
    n = M.shape[0]
    ipr = np.median((vecs[:, 1:] ** 4).sum(0) * n)  # 1: spread evenly, n: one node
    Q, _ = np.linalg.qr(Y)
    overlap = np.median(((Q.T @ vecs[:, 1:]) ** 2).sum(0))  # share of each eigenvector in the indicators' span
    degree_under = np.median((vecs[:, 1:] ** 2 * s[:, None]).sum(0))  # mean degree weighted by |v|^2
    return vals, ipr, overlap, degree_under


def test_lowest_eigenvectors_combinatorial_vs_normalised():
    L, Ln, Y, s, k = _laplacians()
    vals, ipr, overlap, deg = _stats(L, Y, s, k)
    rayleigh = np.median([(Y[:, c] @ L @ Y[:, c]) / Y[:, c].sum() for c in range(k)])
    assert vals[-1] < 0.75 * rayleigh       # lambda_20 well below the community indicators' quotients
    assert ipr > 100                         # localised
    assert deg < 0.6 * s.mean()              # on low-degree nodes
    vals_n, ipr_n, overlap_n, deg_n = _stats(Ln, Y, s, k)
    assert ipr_n < 20 and overlap_n > 5 * overlap and overlap_n > 0.2
    assert abs(deg_n - s.mean()) < 0.2 * s.mean()
