"""GPU stability measure (§4.3, Eq. (12)) and adjusted Rand index against the
oracle.

The adjusted Rand index is an FP64 formula of integer counts summed in the same
order on both sides: equal. gamma(k) composes a float pipeline (the GPU filters
in FP32, the oracle in FP64) before integer labels; on a graph with a clear
structure the labels coincide, so gamma agrees to 1e-9 and peaks at the same k;
lam_k agrees to the count's FP32 rounding (1e-3 relative).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_08863_gb300 import build

    build.build()
    import paper_1509_08863_gb300 as m

    return m


def test_adjusted_rand_matches_oracle(sf, oracle_mod):
    rng = np.random.default_rng(3)
    for n, ka, kb in ((1000, 7, 9), (100_001, 100, 100), (5000, 1, 4)):
        a = rng.integers(0, ka, n).astype(np.int32)
        b = np.where(rng.random(n) < 0.7, a % kb, rng.integers(0, kb, n)).astype(np.int32)
        got = sf.adjusted_rand(torch.as_tensor(a, device="cuda"), torch.as_tensor(b, device="cuda"), ka, kb)
        assert got == oracle_mod.adjusted_rand(a, b)
    with pytest.raises(sf.SpecFiltError):
        sf.adjusted_rand(torch.as_tensor(a, device="cuda"), torch.as_tensor(b, device="cuda"), 1, 2)


def _communities(k, m, seed):
    rng = np.random.default_rng(seed)
    src, dst = [], []
    for c in range(k):
        for i in range(m):
            for j in range(i + 1, m):
                if rng.random() < 0.5:
                    src.append(c * m + i)
                    dst.append(c * m + j)
    for _ in range(12):
        u, v = rng.integers(0, k * m, 2)
        src.append(u)
        dst.append(v)
    return np.array(src, np.int32), np.array(dst, np.int32), rng


def test_stability_matches_oracle(sf, oracle_mod):
    k, m, eta, p, J = 4, 40, 12, 60, 4
    n = k * m
    src, dst, rng = _communities(k, m, 21)
    go = oracle_mod.csr_build(n, src, dst)
    g = sf.csr_build(n, torch.as_tensor(src, device="cuda"), torch.as_tensor(dst, device="cuda"), None)
    th = oracle_mod.lanczos_max(go, 60, rng.standard_normal(n))
    lh = oracle_mod.lambda_hat(th, oracle_mod.strength(go))
    Rc = rng.standard_normal((n, eta)) / np.sqrt(eta)
    Rs = [rng.standard_normal((n, eta)) / np.sqrt(eta) for _ in range(J)]
    gam_o, lk_o = oracle_mod.stability(go, lh, p, Rc, Rs, 2, 6, 50, 7, starts=8)
    gam, lk = sf.stability(g, lh, p, torch.as_tensor(Rc, dtype=torch.float32, device="cuda"),
                           torch.as_tensor(np.stack(Rs), dtype=torch.float32, device="cuda"), 2, 6, 50, 8, 7)
    np.testing.assert_allclose(lk, lk_o, rtol=1e-3)
    np.testing.assert_allclose(gam, gam_o, atol=1e-9)
    assert int(np.argmax(gam)) == k - 2 and gam[k - 2] == pytest.approx(1.0)


def test_stability_automatic_order_matches_oracle_at_that_order(sf, oracle_mod):
    """p_filter = 0: the filters take the order that separates adjacent k
    (their cutoffs' theta gap holds +-2 Jackson widths) while the count keeps
    order p; gamma and lam_k equal the oracle's with the same two orders."""
    k, m, eta, p, J = 4, 40, 12, 30, 3
    n = k * m
    src, dst, rng = _communities(k, m, 23)
    go = oracle_mod.csr_build(n, src, dst)
    g = sf.csr_build(n, torch.as_tensor(src, device="cuda"), torch.as_tensor(dst, device="cuda"), None)
    lh = oracle_mod.lambda_hat(oracle_mod.lanczos_max(go, 60, rng.standard_normal(n)), oracle_mod.strength(go))
    Rc = rng.standard_normal((n, eta)) / np.sqrt(eta)
    Rs = [rng.standard_normal((n, eta)) / np.sqrt(eta) for _ in range(J)]
    gam, lk, used = sf.stability(g, lh, p, torch.as_tensor(Rc, dtype=torch.float32, device="cuda"),
                                 torch.as_tensor(np.stack(Rs), dtype=torch.float32, device="cuda"), 2, 6, 50, 8, 7,
                                 p_filter=0, return_order=True)
    assert used >= p
    th = np.arccos(np.clip(2.0 * np.sort(lk) / lh - 1.0, -1.0, 1.0))
    assert np.all(np.abs(np.diff(th)) * (used + 2) >= 4 * np.pi * (1 - 1e-9))  # the gaps inside [2, 6] resolved
    gam_o, lk_o = oracle_mod.stability(go, lh, p, Rc, Rs, 2, 6, 50, 7, starts=8, p_filter=used)
    np.testing.assert_allclose(lk, lk_o, rtol=1e-3)
    np.testing.assert_allclose(gam, gam_o, atol=1e-9)
