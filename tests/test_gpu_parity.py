"""GPU parity: the CUDA path (through the C ABI) against the CPU FP64 oracle
on the same seeded inputs.

Tolerances:
* CSR (indices and merged weights): bit-exact. Strengths: equal (both sum the
  same FP32 weights in column order in FP64).
* Filtered blocks, FP32 storage: relative Frobenius error <= 1e-5 per
  coefficient set at p = 50 (the stated target); larger p is bounded by
  the FP32 rounding growth 1e-5 * (p / 50)^1.5 and reported.
* Moments: |mu_gpu - mu_oracle| <= 2e-6 * (m + 1) * mu_0 (FP32 blocks, FP64
  reductions); counts derive from them.
* Features: 1e-6 relative per row; adjoint 2e-4 relative (FP32 over p orders).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from helpers import (cliques_edges, dense_laplacian, dense_w, oracle_lambda_hat, random_graph,  # noqa: E402
                     stored_block_error_model)


@pytest.fixture(scope="module")
def sf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_08863_gb300 import build

    build.build()
    import paper_1509_08863_gb300 as m

    return m


def cuda_edges(src, dst, w=None):
    s = torch.as_tensor(np.asarray(src, np.int32), device="cuda")
    d = torch.as_tensor(np.asarray(dst, np.int32), device="cuda")
    ww = None if w is None else torch.as_tensor(np.asarray(w, np.float32), device="cuda")
    return s, d, ww


def build_both(sf, oracle_mod, n, src, dst, w=None):
    w32 = None if w is None else np.asarray(w, np.float32)
    g = sf.csr_build(n, *cuda_edges(src, dst, w32))
    go = oracle_mod.csr_build(n, src, dst, None if w32 is None else w32.astype(np.float64))
    return g, go


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def config1_graph():
    from paper_1509_08863_gb300 import synth

    sizes = synth.community_sizes_equal(1000, 10)
    return synth.sbm_edges(1000, sizes, 16.0, 0.05, seed=1001)


# ------------------------------------------------------------------ CSR
@pytest.mark.parametrize("seed", [0, 1])
def test_csr_bitexact_random_multigraph(sf, oracle_mod, seed):
    n = 777
    src, dst, w = random_graph(n, 6000, seed, connected=False)
    src = np.concatenate([src, src[:500], np.arange(50)]).astype(np.int32)   # duplicates
    dst = np.concatenate([dst, dst[:500], np.arange(50)]).astype(np.int32)   # and self-loops
    w = np.concatenate([w, np.random.default_rng(seed).uniform(0, 3, 500), np.ones(50)]).astype(np.float32)
    g, go = build_both(sf, oracle_mod, n, src, dst, w)
    rp, ci, va, st = [t.cpu().numpy() for t in g.csr()]
    np.testing.assert_array_equal(rp, go.rowptr)
    np.testing.assert_array_equal(ci, go.colidx)
    np.testing.assert_array_equal(va, go.val.astype(np.float32))
    np.testing.assert_array_equal(st, oracle_mod.strength(go))
    assert g.info()[2] is False


def test_csr_order_independent_and_unit_flag(sf, oracle_mod):
    gr = config1_graph()
    g1 = sf.csr_build(gr.n, *cuda_edges(gr.src, gr.dst, gr.w))
    perm = np.random.default_rng(5).permutation(gr.n_edges)
    g2 = sf.csr_build(gr.n, *cuda_edges(gr.dst[perm], gr.src[perm], gr.w[perm]))
    for a, b in zip(g1.csr(), g2.csr()):
        assert torch.equal(a, b)
    go = oracle_mod.csr_build(gr.n, gr.src, gr.dst, gr.w)
    np.testing.assert_array_equal(g1.csr()[1].cpu().numpy(), go.colidx)
    assert g1.info()[2] is True


def test_csr_edge_cases(sf, oracle_mod):
    # no edges, one node
    g = sf.csr_build(1, *cuda_edges(np.zeros(0), np.zeros(0)))
    assert g.info()[:2] == (1, 0)
    # only self-loops and isolated nodes
    g = sf.csr_build(9, *cuda_edges([1, 1, 4], [1, 1, 4]))
    assert g.info()[1] == 0 and list(g.csr()[0].cpu().numpy()) == [0] * 10
    # a hub row far longer than a warp or a tile
    n = 70000
    src = np.zeros(n - 1, np.int32)
    dst = np.arange(1, n, dtype=np.int32)
    g, go = build_both(sf, oracle_mod, n, src, dst)
    np.testing.assert_array_equal(g.csr()[1].cpu().numpy(), go.colidx)
    np.testing.assert_array_equal(g.csr()[0].cpu().numpy(), go.rowptr)


def test_csr_rejects_bad_input(sf):
    with pytest.raises(sf.SpecFiltError) as e:
        sf.csr_build(5, *cuda_edges([0, 1], [1, 5]))
    assert e.value.status == 1
    with pytest.raises(sf.SpecFiltError):
        sf.csr_build(5, *cuda_edges([0, 1], [1, 2], [1.0, -1.0]))
    with pytest.raises(sf.SpecFiltError):
        sf.csr_build(5, *cuda_edges([0, 1], [1, 2], [1.0, float("inf")]))


# ------------------------------------------------------------------ lambda_N
def test_lambda_max_matches_oracle_and_bounds(sf, oracle_mod):
    n = 600
    src, dst, w = random_graph(n, 5000, 3)
    g, go = build_both(sf, oracle_mod, n, src, dst, w)
    v0 = np.random.default_rng(0).standard_normal(n)
    th, lh = sf.lambda_max_estimate(g, 60, torch.as_tensor(v0, device="cuda"))
    tho = oracle_mod.lanczos_max(go, 60, v0)
    lam = np.linalg.eigvalsh(dense_laplacian(dense_w(n, src, np.asarray(dst), np.asarray(w, np.float32))))[-1]
    assert abs(th - tho) <= 1e-9 * tho
    assert abs(th - lam) <= 1e-8 * lam
    assert lam <= lh <= 2 * oracle_mod.strength(go).max() * (1 + 1e-12)
    assert lh == pytest.approx(oracle_mod.lambda_hat(tho, oracle_mod.strength(go)), rel=1e-12)
    # seeded start vector (no v0) converges too
    th2, _ = sf.lambda_max_estimate(g, 60, None, seed=7)
    assert abs(th2 - lam) <= 1e-8 * lam


def test_lambda_max_closed_forms(sf):
    # complete graph K_n and star S_n: lambda_N = n
    for n, (s, d) in [(13, np.triu_indices(13, 1)), (40, (np.zeros(39, int), np.arange(1, 40)))]:
        g = sf.csr_build(n, *cuda_edges(s, d))
        th, _ = sf.lambda_max_estimate(g, n, None, seed=3)
        assert abs(th - n) <= 1e-9 * n


# ------------------------------------------------------------------ filter
def _setup_config1(sf, oracle_mod):
    gr = config1_graph()
    g, go = build_both(sf, oracle_mod, gr.n, gr.src, gr.dst, gr.w)
    lam = np.linalg.eigvalsh(dense_laplacian(dense_w(gr.n, gr.src, gr.dst)))
    from paper_1509_08863_gb300 import synth

    R = synth.gaussian_block(gr.n, 14, seed=2001)
    lh = oracle_lambda_hat(oracle_mod, go, 60, seed=1)
    return gr, g, go, lam, R, lh


@pytest.mark.parametrize("algo", ["forward", "clenshaw"])
@pytest.mark.parametrize("slab", [0, 8, 32])
def test_filter_config1_fp32_within_1e5(sf, oracle_mod, algo, slab):
    gr, g, go, lam, R, lh = _setup_config1(sf, oracle_mod)
    p, k = 50, 10
    a = oracle_mod.cheb_coeffs(lh, lam[k - 1], p, True)  # lambda_c = true lambda_k
    Yo = oracle_mod.cheb_filter(go, lh, a, R)[0]
    opts = sf.Opts(algo=sf.ALGO_FORWARD if algo == "forward" else sf.ALGO_CLENSHAW, slab_cols=slab)
    Y = sf.cheb_filter(g, lh, a, torch.as_tensor(R, dtype=torch.float32, device="cuda"), opts)[0]
    err = rel(Y.cpu().numpy(), Yo)
    assert err <= 1e-5, err


def test_filter_multi_cutoff_ragged(sf, oracle_mod):
    n, n_sig, p = 3001, 37, 23
    src, dst, w = random_graph(n, 20000, 9)
    g, go = build_both(sf, oracle_mod, n, src, dst, w)
    lh = oracle_lambda_hat(oracle_mod, go, 40, seed=2)
    R = np.random.default_rng(4).standard_normal((n, n_sig)) / math.sqrt(n_sig)
    a = oracle_mod.cheb_coeffs(lh, [0.05 * lh, 0.2 * lh, 0.7 * lh], p, True)
    Yo = oracle_mod.cheb_filter(go, lh, a, R)
    Rt = torch.as_tensor(R, dtype=torch.float32, device="cuda")
    for slab in (8, 16, 64):
        Y = sf.cheb_filter(g, lh, a, Rt, sf.Opts(algo=sf.ALGO_FORWARD, slab_cols=slab)).cpu().numpy()
        for c in range(3):
            assert rel(Y[c], Yo[c]) <= 1e-5
        Yc = sf.cheb_filter(g, lh, a, Rt, sf.Opts(algo=sf.ALGO_CLENSHAW, slab_cols=slab)).cpu().numpy()
        for c in range(3):
            assert rel(Yc[c], Yo[c]) <= 1e-5


@pytest.mark.parametrize("p", [0, 1, 2, 3])
def test_filter_low_orders(sf, oracle_mod, p):
    n = 500
    src, dst, w = random_graph(n, 3000, 12)
    g, go = build_both(sf, oracle_mod, n, src, dst, w)
    lh = 2.0 * oracle_mod.strength(go).max()
    R = np.random.default_rng(1).standard_normal((n, 10))
    a = np.random.default_rng(2).standard_normal((2, p + 1))
    Yo = oracle_mod.cheb_filter(go, lh, a, R)
    Rt = torch.as_tensor(R, dtype=torch.float32, device="cuda")
    for algo in (sf.ALGO_FORWARD, sf.ALGO_CLENSHAW):
        Y = sf.cheb_filter(g, lh, a, Rt, sf.Opts(algo=algo)).cpu().numpy()
        for c in range(2):
            assert rel(Y[c], Yo[c]) <= 2e-6


def test_filter_empty_rows_and_bf16_input(sf, oracle_mod):
    n = 1200
    src, dst, w = random_graph(n // 2, 3000, 21)  # upper half of the nodes isolated
    g, go = build_both(sf, oracle_mod, n, src, dst, w)
    lh = 2.0 * oracle_mod.strength(go).max()
    R = np.random.default_rng(3).standard_normal((n, 16)).astype(np.float32)
    Rb_h = torch.as_tensor(R).to(torch.bfloat16)  # rounded on the host
    Rr = Rb_h.double().numpy()  # the values the GPU sees
    Rb = Rb_h.to("cuda")
    a = oracle_mod.cheb_coeffs(lh, 0.3 * lh, 30, True)
    Yo = oracle_mod.cheb_filter(go, lh, a, Rr)[0]
    Y = sf.cheb_filter(g, lh, a, Rb)[0].cpu().numpy()
    assert rel(Y, Yo) <= 1e-5
    # isolated rows: Lt x = -x, so Y_i = sum_j a_j T_j(-1) r_i
    iso = np.arange(n // 2, n)
    fac = np.polynomial.chebyshev.chebval(-1.0, a[0])
    np.testing.assert_allclose(Y[iso], fac * Rr[iso], rtol=1e-5, atol=1e-6)


def test_filter_bf16_storage_error(sf, oracle_mod, record_property):
    """BF16 blocks, FP32 accumulation: the error against the oracle fed the
    BF16-rounded R stays below the stored-block rounding model of
    helpers.stored_block_error_model (u = 2^-8, from the graph's dense
    spectrum); measured on GB300 at about half of it (forward 4.4e-3 against
    7.8e-3, Clenshaw 7.9e-3 against 1.6e-2)."""
    gr, g, go, lam, R, lh = _setup_config1(sf, oracle_mod)
    p = 50
    a = oracle_mod.cheb_coeffs(lh, 0.5 * (lam[9] + lam[10]), p, True)
    Rt = torch.as_tensor(R, dtype=torch.float32, device="cuda")
    Rr = torch.as_tensor(R.astype(np.float32)).to(torch.bfloat16).double().numpy()  # rounded on the host
    Yo_r = oracle_mod.cheb_filter(go, lh, a, Rr)[0]
    for algo, name in ((sf.ALGO_FORWARD, "forward"), (sf.ALGO_CLENSHAW, "clenshaw")):
        Y = sf.cheb_filter(g, lh, a, Rt, sf.Opts(storage=sf.BF16, algo=algo))[0].cpu().numpy()
        err = rel(Y, Yo_r)
        bound = stored_block_error_model(2.0 * lam / lh - 1.0, a[0], 2.0 ** -8, name, False)
        record_property(f"err_bf16_{name}", err)
        record_property(f"bound_bf16_{name}", bound)
        assert err <= bound, (name, err, bound)


@pytest.mark.parametrize("algo", ["forward", "clenshaw"])
def test_filter_f16_storage_error_and_range(sf, oracle_mod, algo, record_property):
    """FP16 blocks (11-bit significand) with the per-slab power-of-two
    prescale: the error against the FP64 oracle (R rounded too) stays below
    the stored-block rounding model (u = 2^-11, input rounding included);
    measured at about half of it (forward 5.8e-4 against 1.0e-3, Clenshaw
    1.0e-3 against 2.1e-3); inputs far outside the FP16 range give the same
    relative error."""
    gr, g, go, lam, R, lh = _setup_config1(sf, oracle_mod)
    p = 50
    a = oracle_mod.cheb_coeffs(lh, 0.5 * (lam[9] + lam[10]), p, True)
    Yo = oracle_mod.cheb_filter(go, lh, a, R)[0]
    A = sf.ALGO_FORWARD if algo == "forward" else sf.ALGO_CLENSHAW
    bound = stored_block_error_model(2.0 * lam / lh - 1.0, a[0], 2.0 ** -11, algo, True)
    record_property(f"bound_f16_{algo}", bound)
    for scale in (1.0, 1e5, 1e-6):
        Rt = torch.as_tensor(R * scale, dtype=torch.float32, device="cuda")
        Y = sf.cheb_filter(g, lh, a, Rt, sf.Opts(storage=sf.F16, algo=A))[0].cpu().numpy() / scale
        assert np.all(np.isfinite(Y))
        err = rel(Y, Yo)
        record_property(f"err_f16_{algo}_scale{scale:g}", err)
        assert err <= bound, (scale, err, bound)


@pytest.mark.parametrize("weighted", [False, True])
def test_direct_kernel_matches_tiled_and_oracle(sf, oracle_mod, weighted):
    """The unstaged sweep kernel sums every row in the same order as the staged
    tiles: filter (both algorithms, several cutoffs) and the adjoint agree bit
    for bit across lane-group widths and storages, moments to FP64 reduction
    order, and the FP32 filter meets the oracle bound. Ragged sizes: N = 3001 (not a multiple of
    the 8-row slices or the tiles), 37 signals (partial last slab)."""
    n, n_sig, p = 3001, 37, 23
    src, dst, w = random_graph(n, 20000, 31)
    g, go = build_both(sf, oracle_mod, n, src, dst, w if weighted else None)
    lh = oracle_lambda_hat(oracle_mod, go, 40, seed=2)
    R = np.random.default_rng(5).standard_normal((n, n_sig)) / math.sqrt(n_sig)
    a = oracle_mod.cheb_coeffs(lh, [0.05 * lh, 0.3 * lh], p, True)
    Yo = oracle_mod.cheb_filter(go, lh, a, R)
    Rt = torch.as_tensor(R, dtype=torch.float32, device="cuda")
    cases = [(sf.F32, s) for s in (8, 16, 32, 64, 128)] + [(sf.BF16, s) for s in (16, 32, 64)] + [(sf.F16, 32)]
    for st, slab in cases:
        for algo in (sf.ALGO_FORWARD, sf.ALGO_CLENSHAW):
            out = []
            for kind in (sf.SWEEP_TILED, sf.SWEEP_DIRECT):
                o = sf.Opts(storage=st, algo=algo, slab_cols=slab, sweep_kernel=kind)
                out.append(sf.cheb_filter(g, lh, a, Rt, o).cpu().numpy())
            assert np.array_equal(out[0], out[1]), (st, slab, algo)
            if st == sf.F32:
                for c in range(2):
                    assert rel(out[1][c], Yo[c]) <= 1e-5
        if st != sf.F16:
            mus = [sf.cheb_moments(g, lh, Rt, p, sf.Opts(storage=st, slab_cols=slab, sweep_kernel=kind))
                   for kind in (sf.SWEEP_TILED, sf.SWEEP_DIRECT)]
            # same blocks; the FP64 moment sums differ only in the order rows reach them
            assert np.all(np.abs(mus[0] - mus[1]) <= 1e-12 * mus[0][0]), (st, slab)
    # the persisting-L2 window changes cache hints only
    yw = [sf.cheb_filter(g, lh, a, Rt, sf.Opts(storage=sf.BF16, slab_cols=32, l2_window=w)).cpu().numpy()
          for w in (0, 1)]
    assert np.array_equal(yw[0], yw[1])
    G = torch.as_tensor(np.random.default_rng(6).standard_normal((n, n_sig)), dtype=torch.float32, device="cuda")
    grads = [sf.cheb_filter_backward(g, lh, a[0], Rt, G, True, sf.Opts(slab_cols=32, sweep_kernel=kind))
             for kind in (sf.SWEEP_TILED, sf.SWEEP_DIRECT)]
    assert torch.equal(grads[0][0], grads[1][0])
    assert np.array_equal(grads[0][1], grads[1][1])
    assert torch.equal(grads[0][2], grads[1][2])


def test_default_slab_on_a_mid_size_graph(sf):
    """A 150k-node graph with 64 FP32 signals: the automatic slab is the whole
    64-column block (38 MB, under the 64 MB budget), where a 16-column slab was
    the default before. Each column's arithmetic does not depend on the slab,
    so the filter (both algorithms, two cutoffs) is bit-identical to 16-column
    slabs, the moments agree to FP64 reduction order and the adjoint to its
    tolerance."""
    from paper_1509_08863_gb300 import synth

    n, n_sig, p = 150_000, 64, 20
    gr = synth.sbm_edges(n, synth.community_sizes_equal(n, 10), 10.0, 0.1, seed=41)
    dev = torch.device("cuda")
    g = sf.csr_build(n, torch.as_tensor(gr.src, device=dev), torch.as_tensor(gr.dst, device=dev), None)
    lh = 2.0 * float((np.bincount(gr.src, minlength=n) + np.bincount(gr.dst, minlength=n)).max())
    a = sf.cheb_coeffs(lh, [0.05 * lh, 0.2 * lh], p, True)
    R = torch.randn(n, n_sig, device="cuda", generator=torch.Generator(device="cuda").manual_seed(3)) / 8.0
    for algo in (sf.ALGO_FORWARD, sf.ALGO_CLENSHAW):
        y_auto = sf.cheb_filter(g, lh, a, R, sf.Opts(algo=algo))
        y_16 = sf.cheb_filter(g, lh, a, R, sf.Opts(algo=algo, slab_cols=16))
        assert torch.equal(y_auto, y_16), algo
    mu_auto = sf.cheb_moments(g, lh, R, p)
    mu_16 = sf.cheb_moments(g, lh, R, p, sf.Opts(slab_cols=16))
    assert np.all(np.abs(mu_auto - mu_16) <= 2e-6 * (np.arange(2 * p + 1) + 1) * mu_auto[0])
    G = torch.randn(n, n_sig, device="cuda", generator=torch.Generator(device="cuda").manual_seed(4))
    gw_a, ga_a, _ = sf.cheb_filter_backward(g, lh, a[0], R, G, False)
    gw_16, ga_16, _ = sf.cheb_filter_backward(g, lh, a[0], R, G, False, sf.Opts(slab_cols=16))
    assert rel(gw_a.cpu().numpy(), gw_16.cpu().numpy()) <= 2e-5
    assert np.all(np.abs(ga_a - ga_16) <= 2e-5 * np.abs(ga_16).max())
    sf.device_check()


# ------------------------------------------------------------------ moments / count
def test_moments_and_counts_match_oracle(sf, oracle_mod):
    from paper_1509_08863_gb300 import synth

    n, eta, p = 2000, 24, 40
    sizes = synth.community_sizes_uniform(n, 8, 100, 400, seed=1)
    gr = synth.sbm_edges(n, sizes, 12.0, 0.1, seed=2)
    g, go = build_both(sf, oracle_mod, n, gr.src, gr.dst, gr.w)
    lh = oracle_lambda_hat(oracle_mod, go, 50, seed=1)
    R = synth.gaussian_block(n, eta, seed=3)
    Rt = torch.as_tensor(R, dtype=torch.float32, device="cuda")
    mu = sf.cheb_moments(g, lh, Rt, p)
    muo = oracle_mod.moments(go, lh, R, 2 * p)
    for m in range(2 * p + 1):
        assert abs(mu[m] - muo[m]) <= 2e-6 * (m + 1) * muo[0], (m, mu[m], muo[m])
    cuts = np.linspace(0.0, 0.2 * lh, 16)
    counts, _ = sf.eigencount(g, lh, Rt, p, cuts, True)
    a = oracle_mod.cheb_coeffs(lh, cuts, p, True)
    co = oracle_mod.eigencount(go, lh, a, R)
    bound = 2e-6 * (2 * p + 1) * muo[0] * np.sum(np.abs(a), axis=1) ** 2
    assert np.all(np.abs(counts - co) <= bound), (counts, co)
    # other slab widths regroup the FP32 row partials: same bound
    mu2 = sf.cheb_moments(g, lh, Rt, p, sf.Opts(slab_cols=8))
    for m in range(2 * p + 1):
        assert abs(mu2[m] - muo[m]) <= 2e-6 * (m + 1) * muo[0]


def test_moments_deterministic(sf, oracle_mod):
    gr = config1_graph()
    g = sf.csr_build(gr.n, *cuda_edges(gr.src, gr.dst, gr.w))
    R = torch.randn(gr.n, 14, device="cuda")
    m1 = sf.cheb_moments(g, 70.0, R, 30)
    m2 = sf.cheb_moments(g, 70.0, R, 30)
    np.testing.assert_array_equal(m1, m2)


def test_dichotomy_finds_gap_on_cliques(sf, oracle_mod):
    k, m, eta, p = 6, 12, 128, 120
    src, dst = cliques_edges(k, m)
    rng = np.random.default_rng(0)
    src = np.concatenate([src, rng.integers(0, k * m, 8)]).astype(np.int32)
    dst = np.concatenate([dst, rng.integers(0, k * m, 8)]).astype(np.int32)
    n = k * m
    g, go = build_both(sf, oracle_mod, n, src, dst)
    lam = np.linalg.eigvalsh(dense_laplacian(dense_w(n, src, dst)))
    lh = oracle_lambda_hat(oracle_mod, go, n, seed=1)
    R = np.random.default_rng(1).standard_normal((n, eta)) / math.sqrt(eta)
    Rt = torch.as_tensor(R, dtype=torch.float32, device="cuda")
    mu = sf.cheb_moments(g, lh, Rt, p)
    lk = sf.dichotomy(mu, p, lh, k - 0.5, True, 40, 1e-9)
    lk_o = oracle_mod.dichotomy(go, lh, p, R, k - 0.5, True, 40, 1e-9)
    assert lam[k - 1] < lk < lam[k] and lam[k - 1] < lk_o < lam[k]
    assert abs(lk - lk_o) <= 0.05 * (lam[k] - lam[k - 1])


# ------------------------------------------------------------------ features
def test_features_match_oracle(sf, oracle_mod):
    rng = np.random.default_rng(8)
    Y = rng.standard_normal((3001, 37)).astype(np.float32)
    Y[[0, 17, 3000]] = 0.0
    Fo = oracle_mod.features(Y.astype(np.float64), True)
    F = sf.features(torch.as_tensor(Y, device="cuda"), True).cpu().numpy()
    nr = np.linalg.norm(Fo, axis=1)
    np.testing.assert_allclose(F, Fo, rtol=0, atol=1e-6 * max(nr.max(), 1))
    assert np.all(F[[0, 17, 3000]] == 0)
    F0 = sf.features(torch.as_tensor(Y, device="cuda"), False).cpu().numpy()
    np.testing.assert_array_equal(F0, Y)


# ------------------------------------------------------------------ adjoint
@pytest.mark.parametrize("ckpt", [1, 3])
def test_backward_matches_oracle(sf, oracle_mod, ckpt):
    n, n_sig, p = 400, 12, 17
    src, dst, w = random_graph(n, 2500, 31)
    g, go = build_both(sf, oracle_mod, n, src, dst, w)
    lh = 2.0 * oracle_mod.strength(go).max()
    rng = np.random.default_rng(5)
    R = rng.standard_normal((n, n_sig)).astype(np.float32)
    G = rng.standard_normal((n, n_sig)).astype(np.float32)
    a = oracle_mod.cheb_coeffs(lh, 0.25 * lh, p, True)[0]
    gv_o, ga_o, gR_o = oracle_mod.cheb_filter_backward(go, lh, a, R.astype(np.float64), G.astype(np.float64), True)
    gv, ga, gR = sf.cheb_filter_backward(g, lh, a, torch.as_tensor(R, device="cuda"), torch.as_tensor(G, device="cuda"),
                                         True, sf.Opts(ckpt_every=ckpt, slab_cols=16))
    assert rel(gv.cpu().numpy(), gv_o) <= 2e-4
    assert rel(ga, ga_o) <= 2e-5
    assert rel(gR.cpu().numpy(), gR_o) <= 2e-5


@pytest.mark.parametrize("slab", [8, 32, 64, 128])
def test_backward_lane_widths_and_unit_weights(sf, oracle_mod, slab):
    """Every lane-group width of the sampled-product kernel (2, 8, 16, 32 lanes
    per row), on a ragged size (N = 1037, 21 signals: a partial slab) and on
    unit weights (the unweighted sweep path)."""
    n, n_sig, p = 1037, 21, 13
    src, dst, _ = random_graph(n, 6000, 37)
    g, go = build_both(sf, oracle_mod, n, src, dst, None)
    lh = 2.0 * oracle_mod.strength(go).max()
    rng = np.random.default_rng(slab)
    R = rng.standard_normal((n, n_sig)).astype(np.float32)
    G = rng.standard_normal((n, n_sig)).astype(np.float32)
    a = oracle_mod.cheb_coeffs(lh, 0.3 * lh, p, True)[0]
    gv_o, ga_o, gR_o = oracle_mod.cheb_filter_backward(go, lh, a, R.astype(np.float64), G.astype(np.float64), True)
    gv, ga, gR = sf.cheb_filter_backward(g, lh, a, torch.as_tensor(R, device="cuda"), torch.as_tensor(G, device="cuda"),
                                         True, sf.Opts(slab_cols=slab))
    assert rel(gv.cpu().numpy(), gv_o) <= 2e-4
    assert rel(ga, ga_o) <= 2e-5
    assert rel(gR.cpu().numpy(), gR_o) <= 2e-5


def test_backward_checkpoint_equals_store(sf, oracle_mod):
    n, n_sig, p = 900, 20, 30
    src, dst, w = random_graph(n, 6000, 41)
    g, go = build_both(sf, oracle_mod, n, src, dst, w)
    lh = 2.0 * oracle_mod.strength(go).max()
    R = torch.randn(n, n_sig, device="cuda")
    G = torch.randn(n, n_sig, device="cuda")
    a = np.random.default_rng(0).standard_normal(p + 1) * 0.1
    out1 = sf.cheb_filter_backward(g, lh, a, R, G, True, sf.Opts(ckpt_every=1))
    out2 = sf.cheb_filter_backward(g, lh, a, R, G, True, sf.Opts(ckpt_every=6))
    assert torch.equal(out1[0], out2[0]) and torch.equal(out1[2], out2[2])
    np.testing.assert_array_equal(out1[1], out2[1])


def test_autograd_function(sf, oracle_mod):
    n, n_sig, p = 300, 8, 12
    src, dst, w = random_graph(n, 1500, 51)
    g, go = build_both(sf, oracle_mod, n, src, dst, w)
    lh = 2.0 * oracle_mod.strength(go).max()
    val = g.csr()[2].clone().requires_grad_(True)
    coeffs = torch.tensor(oracle_mod.cheb_coeffs(lh, 0.3 * lh, p, True)[0], dtype=torch.float64,
                          requires_grad=True)
    R = torch.randn(n, n_sig, device="cuda", requires_grad=True)
    Y = sf.ChebFilter(val, coeffs, R, g, lh)
    G = torch.randn_like(Y)
    (Y * G).sum().backward()
    gv_o, ga_o, gR_o = oracle_mod.cheb_filter_backward(go, lh, coeffs.detach().numpy(),
                                                       R.detach().cpu().double().numpy(),
                                                       G.cpu().double().numpy(), True)
    assert rel(val.grad.cpu().numpy(), gv_o) <= 2e-4
    assert rel(coeffs.grad.numpy(), ga_o) <= 2e-5
    assert rel(R.grad.cpu().numpy(), gR_o) <= 2e-5


# ------------------------------------------------------------------ batches
def test_batched_matches_oracle_and_single_launches(sf, oracle_mod):
    from paper_1509_08863_gb300 import synth

    graphs, ks = synth.batched_sbm(5, seed=77, n_lo=300, n_hi=2500, k_lo=2, k_hi=6)
    gs, gos, lams = [], [], []
    for gr in graphs:
        g, go = build_both(sf, oracle_mod, gr.n, gr.src, gr.dst, gr.w)
        gs.append(g)
        gos.append(go)
        lams.append(oracle_lambda_hat(oracle_mod, go, 40, seed=1))
    b = sf.batch_build(gs)
    n_tot, nnz_tot, ng, offs = b.info()
    assert ng == 5 and n_tot == sum(gr.n for gr in graphs)
    p, n_sig = 30, 32
    coeffs = np.stack([oracle_mod.cheb_coeffs(lams[i], (0.02 + 0.03 * i) * lams[i], p, True)[0] for i in range(5)])
    R = np.random.default_rng(9).standard_normal((n_tot, n_sig)) / math.sqrt(n_sig)
    Rt = torch.as_tensor(R, dtype=torch.float32, device="cuda")
    for algo in (sf.ALGO_CLENSHAW, sf.ALGO_FORWARD):
        opts = sf.Opts(algo=algo, slab_cols=32)
        Y = sf.cheb_filter_batched(b, lams, coeffs, Rt, opts)
        for i in range(5):
            sl = slice(int(offs[i]), int(offs[i + 1]))
            Yo = oracle_mod.cheb_filter(gos[i], lams[i], coeffs[i], R[sl])[0]
            assert rel(Y[sl].cpu().numpy(), Yo) <= 1e-5
            Ys = sf.cheb_filter(gs[i], lams[i], coeffs[i], Rt[sl].contiguous(), opts)[0]
            assert torch.equal(Ys, Y[sl])  # same per-row arithmetic, bit for bit


def test_batched_device_tables_under_cuda_graph(sf, oracle_mod):
    from paper_1509_08863_gb300 import synth

    graphs, _ = synth.batched_sbm(4, seed=91, n_lo=400, n_hi=1500, k_lo=2, k_hi=5)
    gs = [sf.csr_build(gr.n, *cuda_edges(gr.src, gr.dst, gr.w)) for gr in graphs]
    lams = [sf.lambda_max_estimate(g, 30, None, seed=1)[1] for g in gs]
    b = sf.batch_build(gs)
    n_tot = b.info()[0]
    p = 20
    coeffs = np.stack([sf.cheb_coeffs(lams[i], 0.1 * lams[i], p, True)[0] for i in range(4)])
    R = torch.randn(n_tot, 16, device="cuda")
    for st in (sf.F32, sf.BF16):
        opts = sf.Opts(storage=st, slab_cols=16 if st == sf.F32 else 32)
        Yref = sf.cheb_filter_batched(b, lams, coeffs, R, opts)
        tol_d = torch.as_tensor(2.0 / np.array(lams), dtype=torch.float64, device="cuda")
        coef_d = torch.as_tensor(coeffs, dtype=torch.float32, device="cuda")
        Y = torch.empty_like(Yref)
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            sf.cheb_filter_batched_dev(b, tol_d, coef_d, R, Y, opts)
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        assert torch.equal(Y, Yref)
        Y.zero_()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            sf.cheb_filter_batched_dev(b, tol_d, coef_d, R, Y, opts)
        for _ in range(2):
            Y.zero_()
            graph.replay()
            torch.cuda.synchronize()
            assert torch.equal(Y, Yref)


# ------------------------------------------------------------------ misc
def test_argument_errors(sf):
    gr = config1_graph()
    g = sf.csr_build(gr.n, *cuda_edges(gr.src, gr.dst))
    R = torch.randn(gr.n, 4, device="cuda")
    with pytest.raises(sf.SpecFiltError):
        sf.cheb_filter(g, -1.0, np.ones((1, 3)), R)
    with pytest.raises(sf.SpecFiltError):
        sf.cheb_moments(g, 10.0, R, 3, sf.Opts(storage=sf.F16))  # moments need FP32 or BF16 blocks
    with pytest.raises(sf.SpecFiltError):
        sf.cheb_filter(g, 10.0, np.ones((1, 3)), R, sf.Opts(storage=7))
    with pytest.raises(sf.SpecFiltError):
        sf.cheb_filter(g, 10.0, np.array([[1.0, float("nan")]]), R)
    with pytest.raises(sf.SpecFiltError):
        sf.cheb_filter(g, 10.0, np.ones((1, 3)), R, sf.Opts(slab_cols=12))


def test_fault_reports_without_fault(sf, oracle_mod):
    """Host-visible failures: lam_max below the spectrum is caught by the
    moment sweep's growth check, NaN signals by its finiteness check, and a
    request larger than the device memory returns SF_ERR_OOM."""
    gr = config1_graph()
    g = sf.csr_build(gr.n, *cuda_edges(gr.src, gr.dst))
    _, lh = sf.lambda_max_estimate(g, 60, None, seed=1)
    R = torch.randn(gr.n, 16, device="cuda")
    with pytest.raises(sf.SpecFiltError) as e:
        sf.cheb_moments(g, 0.5 * lh, R, 60)
    assert e.value.status == 5
    Rn = R.clone()
    Rn[3, 2] = float("nan")
    with pytest.raises(sf.SpecFiltError) as e:
        sf.cheb_moments(g, lh, Rn, 10)
    assert e.value.status == 5
    sf.cheb_moments(g, lh, R, 10)  # the library stays usable
    n = 100_000
    big = sf.csr_build(n, *cuda_edges(np.arange(n - 1), np.arange(1, n)))
    Rb = torch.randn(n, 64, device="cuda")
    with pytest.raises(sf.SpecFiltError) as e:  # (p + 1) stored blocks of 25.6 MB: ~2.6 TB
        sf.cheb_filter_backward(big, 4.0, np.full(100_001, 1e-3), Rb, Rb, False, sf.Opts(ckpt_every=1))
    assert e.value.status == 3
    sf.cheb_moments(g, lh, R, 10)


def test_autotune_and_profile(sf, oracle_mod):
    gr = config1_graph()
    g = sf.csr_build(gr.n, *cuda_edges(gr.src, gr.dst))
    best = sf.autotune(g, 14, sf.F32, 1)
    assert best.slab_cols in (8, 16)
    R = torch.randn(gr.n, 14, device="cuda")
    sf.profile_begin()
    n0 = sf.launch_count()
    sf.cheb_filter(g, 70.0, np.ones((1, 11)) * 0.1, R, best)
    n_l, ms, by = sf.profile_end()
    assert n_l == 10 and ms > 0 and by > 0
    assert sf.launch_count() - n0 >= 12


def test_gather_ceiling_diagnostic(sf):
    r = sf.gather_ceiling(100_000, 64, 32, 2)
    assert np.isfinite(r) and r > 1e9  # rows per second
    r0 = sf.gather_rate(100_000, 64, 32, 2, write_rows=False)
    assert np.isfinite(r0) and r0 > 1e9
    for bad in ((0, 64, 32), (1000, 48, 32), (1000, 64, 30), (1000, 64, 0)):
        with pytest.raises(sf.SpecFiltError):
            sf.gather_ceiling(*bad, 1)
        with pytest.raises(sf.SpecFiltError):
            sf.gather_rate(*bad, 1, write_rows=False)


def test_normalized_laplacian_matches_oracle(sf, oracle_mod):
    """The normalised graph (footnote of §2.1): weights equal the oracle's
    rounded to FP32, unit diagonal (0 for the isolated node), lam_max <= 2 (= 2
    on a bipartite graph), filter and moments within the FP32 bounds of the
    oracle's explicit-diagonal filter; the adjoint and set_values refuse it."""
    n, n_sig, p = 2001, 21, 40
    src, dst, w = random_graph(n - 1, 16000, 41)  # node n - 1 isolated
    g, go = build_both(sf, oracle_mod, n, src, dst, w)
    gn = g.normalized()
    gno = oracle_mod.normalize(go)
    rp, ci, va, st = gn.csr()
    np.testing.assert_array_equal(va.cpu().numpy(), gno.val.astype(np.float32))
    np.testing.assert_array_equal(st.cpu().numpy(), gno.diag)
    th, lh_gpu = sf.lambda_max_estimate(gn, 80, None, seed=4)
    assert th <= 2.0 + 1e-9 and lh_gpu <= 2.0
    lh = 2.0  # the normalised spectrum lies in [0, 2]: the closed-form bound, given to both sides
    R = np.random.default_rng(8).standard_normal((n, n_sig)) / math.sqrt(n_sig)
    Rt = torch.as_tensor(R, dtype=torch.float32, device="cuda")
    a = oracle_mod.cheb_coeffs(lh, [0.2 * lh, 0.5 * lh], p, True)
    Yo = oracle_mod.cheb_filter(gno, lh, a, R)
    for algo in (sf.ALGO_FORWARD, sf.ALGO_CLENSHAW):
        Y = sf.cheb_filter(gn, lh, a, Rt, sf.Opts(algo=algo)).cpu().numpy()
        for c in range(2):
            assert rel(Y[c], Yo[c]) <= 1e-5
    # bipartite (a star): the normalised spectrum reaches 2
    m = 50
    gs = sf.csr_build(m, *cuda_edges(np.zeros(m - 1, int), np.arange(1, m)))
    th_s, _ = sf.lambda_max_estimate(gs.normalized(), m, None, seed=1)
    assert abs(th_s - 2.0) <= 1e-6  # the weights 1/sqrt(s_i s_j) are rounded to FP32
    with pytest.raises(sf.SpecFiltError):
        sf.cheb_filter_backward(gn, lh, a[0], Rt, Rt, False)
    with pytest.raises(sf.SpecFiltError):
        gn.set_values(va)


def test_bounded_wait_gives_up_without_fault(sf, oracle_mod):
    """A wait that can never be satisfied gives up after its poll budget, the
    host reads SF_ERR_TIMEOUT, the flag clears, and the context keeps working."""
    sf.selftest_bounded_wait(2000)
    with pytest.raises(sf.SpecFiltError) as e:
        sf.device_check()
    assert e.value.status == 4  # SF_ERR_TIMEOUT
    sf.device_check()  # cleared
    gr = config1_graph()
    g = sf.csr_build(gr.n, *cuda_edges(gr.src, gr.dst))
    _, lh = sf.lambda_max_estimate(g, 30, None, seed=1)
    R = torch.ones((gr.n, 8), device="cuda")
    Y = sf.cheb_filter(g, lh, sf.cheb_coeffs(lh, 0.3 * lh, 10, True), R)
    sf.device_check()
    assert torch.isfinite(Y).all()


# ------------------------------------------------------------------ persistent batch sweep
def _small_batch(sf, oracle_mod, n_graphs, seed):
    from paper_1509_08863_gb300 import synth

    graphs, _ = synth.batched_sbm(n_graphs, seed=seed, n_lo=300, n_hi=2500, k_lo=2, k_hi=6)
    gs, gos, lams = [], [], []
    for gr in graphs:
        g, go = build_both(sf, oracle_mod, gr.n, gr.src, gr.dst, gr.w)
        gs.append(g)
        gos.append(go)
        lams.append(oracle_lambda_hat(oracle_mod, go, 40, seed=1))
    return graphs, gs, gos, lams, sf.batch_build(gs)


def test_batched_persistent_equals_per_order_launches(sf, oracle_mod):
    """One persistent launch for all orders computes every row with the same
    operations as one launch per order: bit-identical outputs for every
    storage and algorithm, on a batch whose 32768-row sorting window spans
    all 23 graphs (tiles straddle graph boundaries), and within 1e-5 of the
    oracle with several cutoffs per graph (FP32)."""
    graphs, gs, gos, lams, b = _small_batch(sf, oracle_mod, 23, seed=123)
    n_tot, _, ng, offs = b.info()
    p, n_sig = 25, 24
    cuts = np.array([0.03, 0.1, 0.3])
    coeffs3 = np.stack([oracle_mod.cheb_coeffs(lams[i], cuts * lams[i], p, True) for i in range(ng)])
    R = np.random.default_rng(4).standard_normal((n_tot, n_sig)) / math.sqrt(n_sig)
    Rt = torch.as_tensor(R, dtype=torch.float32, device="cuda")
    for st, algo, slab in ((sf.F32, sf.ALGO_CLENSHAW, 16), (sf.F32, sf.ALGO_FORWARD, 8), (sf.BF16, sf.ALGO_FORWARD, 32),
                           (sf.BF16, sf.ALGO_CLENSHAW, 16), (sf.F16, sf.ALGO_FORWARD, 32)):
        outs = []
        for kind in (sf.SWEEP_TILED, sf.SWEEP_PERSISTENT):
            o = sf.Opts(storage=st, algo=algo, slab_cols=slab, sweep_kernel=kind)
            outs.append(sf.cheb_filter_batched(b, lams, coeffs3[:, 1, :], Rt, o))
        sf.device_check()
        assert torch.equal(outs[0], outs[1]), (st, algo, slab)
    for kind in (sf.SWEEP_TILED, sf.SWEEP_PERSISTENT):
        Y = sf.cheb_filter_batched_multi(b, lams, coeffs3, Rt, sf.Opts(algo=sf.ALGO_FORWARD, sweep_kernel=kind))
        if kind == sf.SWEEP_TILED:
            Yt = Y
        else:
            assert torch.equal(Y, Yt)
    Yc = sf.cheb_filter_batched_multi(b, lams, coeffs3, Rt, sf.Opts(algo=sf.ALGO_CLENSHAW,
                                                                     sweep_kernel=sf.SWEEP_PERSISTENT))
    for i in range(ng):
        sl = slice(int(offs[i]), int(offs[i + 1]))
        Yo = oracle_mod.cheb_filter(gos[i], lams[i], coeffs3[i], R[sl])
        for c in range(3):
            assert rel(Yt[c][sl].cpu().numpy(), Yo[c]) <= 1e-5, (i, c)
            assert rel(Yc[c][sl].cpu().numpy(), Yo[c]) <= 1e-5, (i, c)


@pytest.mark.parametrize("n_graphs,n_lo,n_hi", [(40, 3000, 8000), (60, 4000, 8000), (60, 8000, 16000)])
def test_batched_persistent_multi_tile_items(sf, n_graphs, n_lo, n_hi):
    """Batches of about 220k, 380k and 760k rows, large enough that the
    persistent sweep's work items hold several tiles (its claim of the next
    item and the counter poll then happen mid-item): bit-identical to one
    launch per order, forward with two cutoffs in BF16 and Clenshaw in FP32."""
    from paper_1509_08863_gb300 import synth

    graphs, _ = synth.batched_sbm(n_graphs, 777 + n_graphs, n_lo=n_lo, n_hi=n_hi, d_lo=8.0, d_hi=16.0)
    dev = torch.device("cuda")
    gs = [sf.csr_build(gr.n, torch.as_tensor(gr.src, device=dev), torch.as_tensor(gr.dst, device=dev), None)
          for gr in graphs]
    # 2 max_i s_i bounds lambda_N (unit weights: s_i <= the edge list's count of i as either endpoint)
    lams = [2.0 * float((np.bincount(gr.src, minlength=gr.n) + np.bincount(gr.dst, minlength=gr.n)).max())
            for gr in graphs]
    b = sf.batch_build(gs)
    n_tot = b.info()[0]
    p = 12
    coeffs2 = np.stack([np.stack([sf.cheb_coeffs(lams[i], c * lams[i], p, True)[0] for c in (0.05, 0.2)])
                        for i in range(len(gs))])
    R = torch.randn(n_tot, 32, device="cuda", generator=torch.Generator(device="cuda").manual_seed(n_graphs))
    for st, algo in ((sf.BF16, sf.ALGO_FORWARD), (sf.F32, sf.ALGO_CLENSHAW)):
        outs = [sf.cheb_filter_batched_multi(b, lams, coeffs2, R, sf.Opts(storage=st, algo=algo, sweep_kernel=kind))
                for kind in (sf.SWEEP_TILED, sf.SWEEP_PERSISTENT)]
        sf.device_check()
        assert torch.equal(outs[0], outs[1]), (st, algo)


def test_batched_persistent_under_cuda_graph(sf, oracle_mod):
    graphs, gs, gos, lams, b = _small_batch(sf, oracle_mod, 6, seed=321)
    n_tot = b.info()[0]
    p = 17
    coeffs = np.stack([oracle_mod.cheb_coeffs(lams[i], 0.1 * lams[i], p, True)[0] for i in range(len(gs))])
    R = torch.randn(n_tot, 32, device="cuda")
    opts = sf.Opts(storage=sf.BF16, slab_cols=32, sweep_kernel=sf.SWEEP_PERSISTENT)
    Yref = sf.cheb_filter_batched(b, lams, coeffs, R, sf.Opts(storage=sf.BF16, slab_cols=32))
    tol_d = torch.as_tensor(2.0 / np.array(lams), dtype=torch.float64, device="cuda")
    coef_d = torch.as_tensor(coeffs, dtype=torch.float32, device="cuda")
    Y = torch.empty_like(Yref)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        sf.cheb_filter_batched_dev(b, tol_d, coef_d, R, Y, opts)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    assert torch.equal(Y, Yref)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        sf.cheb_filter_batched_dev(b, tol_d, coef_d, R, Y, opts)
    for _ in range(2):
        Y.zero_()
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(Y, Yref)
    sf.device_check()


def test_arrival_wait_gives_up_without_fault(sf, oracle_mod):
    """The persistent batch sweep's wait for a graph's previous order gives up
    after its poll budget (a counter nothing increments), the host reads
    SF_ERR_TIMEOUT, the word clears, and the next batched call works."""
    sf.selftest_arrival_wait(500)
    with pytest.raises(sf.SpecFiltError) as e:
        sf.device_check()
    assert e.value.status == 4
    sf.device_check()
    graphs, gs, gos, lams, b = _small_batch(sf, oracle_mod, 3, seed=7)
    n_tot = b.info()[0]
    coeffs = np.stack([oracle_mod.cheb_coeffs(lams[i], 0.2 * lams[i], 9, True)[0] for i in range(3)])
    Y = sf.cheb_filter_batched(b, lams, coeffs, torch.ones((n_tot, 8), device="cuda"),
                               sf.Opts(sweep_kernel=sf.SWEEP_PERSISTENT))
    sf.device_check()
    assert torch.isfinite(Y).all()
