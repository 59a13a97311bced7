"""CPU checks of the seeded synthetic inputs against the recipe they state:
community sizes, the SBM's mean degree and share of edges between
communities, consistent (permuted) labels, the kNN mixture's edges and
weights, the N(0, 1/eta) signal blocks, and determinism per seed."""
import numpy as np
import pytest

from paper_1509_08863_gb300 import synth


def test_community_sizes():
    s = synth.community_sizes_equal(1003, 10)
    assert s.sum() == 1003 and s.max() - s.min() <= 1
    u = synth.community_sizes_uniform(100_000, 20, 2000, 8000, seed=5)
    assert u.sum() == 100_000 and u.min() >= 1 and len(u) == 20
    assert np.array_equal(u, synth.community_sizes_uniform(100_000, 20, 2000, 8000, seed=5))
    # the draw is uniform in [lo, hi] before the rescaling to n: the spread survives it
    assert u.max() / u.min() > 1.5


def test_sbm_degree_mixing_and_labels():
    n, k, deg, eps = 20_000, 10, 16.0, 0.1
    sizes = synth.community_sizes_equal(n, k)
    gr = synth.sbm_edges(n, sizes, deg, eps, seed=7)
    m = len(gr.src)
    assert abs(2.0 * m / n - deg) / deg < 0.03  # expected mean degree (each undirected edge listed once)
    intra = float((sizes * (sizes - 1)).sum()) / 2.0
    inter = (float(n) * n - float((sizes ** 2).sum())) / 2.0
    expected = eps * inter / (intra + eps * inter)
    lab = gr.labels
    assert abs(np.mean(lab[gr.src] != lab[gr.dst]) - expected) < 0.01
    assert np.array_equal(np.sort(np.bincount(lab, minlength=k)), np.sort(sizes))
    assert len(np.unique(lab[: n // k])) > 1  # node ids are permuted: no block of consecutive ids
    again = synth.sbm_edges(n, sizes, deg, eps, seed=7)
    assert np.array_equal(gr.src, again.src) and np.array_equal(gr.dst, again.dst)
    assert gr.src.dtype == np.int32 and gr.w.dtype == np.float32 and np.all(gr.w == 1.0)


def test_sbm_share_between_communities_at_the_benchmark_parameters():
    # 100 equal communities, c_out/c_in = 0.08: about 89% of the edges join different communities
    k, eps = 100, 0.08
    share = eps * (k - 1) / (1 + eps * (k - 1))
    assert abs(share - 0.888) < 0.001
    n = 50_000
    gr = synth.sbm_edges(n, synth.community_sizes_equal(n, k), 30.0, eps, seed=3)
    assert abs(np.mean(gr.labels[gr.src] != gr.labels[gr.dst]) - share) < 0.01


def test_gaussian_block():
    R = synth.gaussian_block(200_000, 8, seed=11)
    assert R.shape == (200_000, 8) and R.dtype == np.float64
    assert abs(R.mean()) < 3e-3
    assert abs(R.var() - 1.0 / 8) / (1.0 / 8) < 0.01
    assert np.array_equal(R, synth.gaussian_block(200_000, 8, seed=11))
    assert not np.array_equal(R[:100], synth.gaussian_block(100, 8, seed=12))


def test_knn_mixture_edges():
    pytest.importorskip("scipy")
    n, kk, sigma = 2000, 5, 1.0
    src, dst, w, labels, pts = synth.knn_mixture_edges(n, 3, 4, kk, sigma, 3.0, seed=9)
    assert np.all(src != dst)
    assert np.all(np.bincount(src, minlength=n) == kk)  # K neighbours per point
    d2 = ((pts[src] - pts[dst]) ** 2).sum(1)
    np.testing.assert_allclose(w, np.exp(-d2 / sigma ** 2), rtol=1e-6)
    assert np.all((w > 0) & (w <= 1)) and labels.min() >= 0 and labels.max() < 3
    # each listed neighbour is among the K nearest of its source
    i = 17
    order = np.argsort(((pts - pts[i]) ** 2).sum(1))[1:kk + 1]
    assert set(dst[src == i]) == set(order)


def test_batched_sbm():
    graphs, ks = synth.batched_sbm(4, seed=100, n_lo=500, n_hi=900, k_lo=2, k_hi=5)
    assert len(graphs) == 4 and np.all((ks >= 2) & (ks <= 5))
    again, ks2 = synth.batched_sbm(4, seed=100, n_lo=500, n_hi=900, k_lo=2, k_hi=5)
    assert np.array_equal(ks, ks2)
    for g, gr in enumerate(graphs):
        assert 500 <= gr.n <= 900
        assert np.array_equal(gr.src, again[g].src) and np.array_equal(gr.dst, again[g].dst)
        sizes = synth.community_sizes_equal(gr.n, int(ks[g]))
        assert np.array_equal(np.sort(np.bincount(gr.labels)), np.sort(sizes))
        assert gr.src.max() < gr.n and gr.dst.max() < gr.n
