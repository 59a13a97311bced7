"""Column sharding over two CPU ranks (gloo): the host logic of the
multi-GPU path -- column partition, moment all-reduce, row-normalisation
all-reduce -- checked against single-process oracle results. The per-rank
compute is the oracle's; on GPUs it is the library's."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, root):
    import sys

    sys.path.insert(0, root)
    sys.path.insert(0, os.path.join(root, "tests"))
    import oracle
    from helpers import random_graph
    from paper_1509_08863_gb300 import sharded

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        n, n_sig, p = 150, 13, 12
        src, dst, w = random_graph(n, 700, 17)
        g = oracle.csr_build(n, src, dst, w)
        lam = 2.0 * oracle.strength(g).max()
        R = np.random.default_rng(3).standard_normal((n, n_sig)) / np.sqrt(n_sig)
        # every column exactly once
        parts = [sharded.column_shard(n_sig, world, r) for r in range(world)]
        cols = np.concatenate([np.arange(a, b) for a, b in parts])
        assert np.array_equal(cols, np.arange(n_sig))
        c0, c1 = sharded.column_shard(n_sig, world, rank)
        Rl = np.ascontiguousarray(R[:, c0:c1])
        # moments: sum over ranks == moments of the whole block
        mu = sharded.combine_moments(oracle.moments(g, lam, Rl, 2 * p))
        mu_full = oracle.moments(g, lam, R, 2 * p)
        np.testing.assert_allclose(mu, mu_full, rtol=1e-12, atol=1e-12 * mu_full[0])
        # counts and dichotomy agree on every rank
        a = oracle.cheb_coeffs(lam, [0.1 * lam, 0.3 * lam], p, True)
        np.testing.assert_allclose(oracle.count_from_moments(mu, a), oracle.eigencount(g, lam, a, R), rtol=1e-10)
        # features: row norms over all columns
        Yl = oracle.cheb_filter(g, lam, a[:1], Rl)[0]
        F = sharded.normalize_rows_sharded(Yl, lambda Y: np.sum(Y * Y, axis=1),
                                           lambda Y, tot: Y / np.sqrt(tot)[:, None])
        Ffull = oracle.features(oracle.cheb_filter(g, lam, a[:1], R)[0], True)
        np.testing.assert_allclose(F, Ffull[:, c0:c1], rtol=1e-12, atol=1e-14)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_column_sharded_moments_and_features_gloo(world):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    mp.spawn(_worker, args=(world, _free_port(), root), nprocs=world, join=True)


def test_column_shard_edge_cases():
    from paper_1509_08863_gb300 import sharded

    assert sharded.column_shard(5, 8, 7) == (5, 5)  # more ranks than columns: empty shards
    assert sharded.column_shard(128, 4, 3) == (96, 128)
    with pytest.raises(ValueError):
        sharded.column_shard(10, 2, 2)
