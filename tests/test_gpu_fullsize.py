"""GPU parity at the benchmark's full sizes, in the launch configuration the
benchmark times (autotuned tiles, the same storage and algorithms), against
the FP64 oracle on sampled outputs it can compute: signal columns are
independent, so the oracle filters a few columns of R over the whole graph
and the GPU result's matching columns must agree.

Bounds (relative Frobenius error per column against FP64):
* FP32 blocks: 1e-5 (p / 50)^1.5 (FP32 rounding growing through the
  recurrence; 1e-5 is the stated bound at p = 50);
* BF16 blocks, forward recurrence, 1M-node SBM at p = 200: 2^-8 sqrt(p) =
  0.055, 1.7-1.9x the errors measured on GB300 (0.030 and 0.032 on the two
  columns);
* BF16 blocks on the batch: the smallest graph against the stored-block
  rounding model of helpers.stored_block_error_model (its dense spectrum);
  the two large graphs, whose spectra are out of reach, against 5e-3, 2x the
  errors measured on GB300 (2.5e-3).
"""
import math

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


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def oracle_lam(oracle_mod, go, iters, seed):
    from helpers import oracle_lambda_hat

    return oracle_lambda_hat(oracle_mod, go, iters, seed)


def test_sbm1m_filter_and_moments_column_sample(sf, oracle_mod, record_property):
    import bench

    wl = bench.WORKLOADS["sbm1m"]
    gr, R = bench.make_inputs(wl)
    n, p = wl["n"], wl["p"]
    dev = torch.device("cuda")
    g = sf.csr_build(n, torch.as_tensor(gr.src, device=dev), torch.as_tensor(gr.dst, device=dev), None)
    go = oracle_mod.csr_build(n, gr.src, gr.dst, gr.w)
    # lam_hat from the oracle's Lanczos, the cutoff at 0.18 lam_hat (about the workload's lambda_k):
    # the same inputs on both sides
    lh = oracle_lam(oracle_mod, go, 40, seed=11)
    a = oracle_mod.cheb_coeffs(lh, 0.18 * lh, p, True)
    Rt = torch.as_tensor(R, dtype=torch.float32, device=dev)
    tuned = sf.autotune(g, wl["R"], sf.BF16, 1)
    opts = sf.Opts(storage=sf.BF16, slab_cols=tuned.slab_cols, block_warps=tuned.block_warps,
                   carveout_pct=tuned.carveout_pct, l2_window=tuned.l2_window, sweep_kernel=tuned.sweep_kernel)
    cols = [0, 77]
    Yo = oracle_mod.cheb_filter(go, lh, a, np.ascontiguousarray(R[:, cols]))[0]
    Ybf = sf.cheb_filter(g, lh, a, Rt, opts)[0][:, cols].cpu().numpy()
    Y32 = sf.cheb_filter(g, lh, a, Rt, sf.Opts(storage=sf.F32))[0][:, cols].cpu().numpy()
    for c in range(len(cols)):
        record_property(f"err_f32_col{cols[c]}", rel(Y32[:, c], Yo[:, c]))
        record_property(f"err_bf16_col{cols[c]}", rel(Ybf[:, c], Yo[:, c]))
        assert rel(Y32[:, c], Yo[:, c]) <= 1e-5 * (p / 50) ** 1.5
        assert rel(Ybf[:, c], Yo[:, c]) <= 2.0 ** -8 * math.sqrt(p)
    # the moment sweep on a column sample: moments are sums over columns
    mu_s = sf.cheb_moments(g, lh, Rt[:, cols].contiguous(), 6)
    mu_o = oracle_mod.moments(go, lh, np.ascontiguousarray(R[:, cols]), 12)
    for m in range(13):
        assert abs(mu_s[m] - mu_o[m]) <= 2e-6 * (m + 1) * mu_o[0]


def test_knn200k_adjoint_column_sample(sf, oracle_mod):
    """Reverse mode on the full 10-NN graph, two signal columns (the gradients
    are sums over columns, so a two-column run is an exact sub-problem)."""
    import bench
    from paper_1509_08863_gb300 import synth

    wl = bench.WORKLOADS["knn200k"]
    n, p = wl["n"], wl["p"]
    src, dst, w, _, _ = synth.knn_mixture_edges(n, wl["k"], wl["dim"], wl["knn"], wl["sigma"], 3.0, wl["graph_seed"])
    dev = torch.device("cuda")
    g = sf.csr_build(n, torch.as_tensor(src, device=dev), torch.as_tensor(dst, device=dev),
                     torch.as_tensor(w, device=dev))
    go = oracle_mod.csr_build(n, src, dst, w.astype(np.float64))
    lh = oracle_lam(oracle_mod, go, 60, seed=11)
    R = synth.gaussian_block(n, 2, wl["r_seed"]).astype(np.float32)
    G = synth.standard_normal_block(n, 2, wl["g_seed"]).astype(np.float32)
    a = oracle_mod.cheb_coeffs(lh, 0.02 * lh, p, True)[0]
    gv, ga, gR = sf.cheb_filter_backward(g, lh, a, torch.as_tensor(R, device=dev), torch.as_tensor(G, device=dev),
                                         True)
    gv_o, ga_o, gR_o = oracle_mod.cheb_filter_backward(go, lh, a, R.astype(np.float64), G.astype(np.float64), True)
    assert rel(gv.cpu().numpy(), gv_o) <= 1e-3
    assert rel(ga, ga_o) <= 1e-4
    assert rel(gR.cpu().numpy(), gR_o) <= 1e-4


def test_batch256_sampled_graphs(sf, oracle_mod, record_property):
    """The batched filter over all 256 graphs; three graphs (smallest,
    largest, one in between) checked on two columns against the oracle."""
    import bench
    from paper_1509_08863_gb300 import synth

    wl = bench.WORKLOADS["batch256"]
    p, eta = wl["p"], wl["R"]
    graphs, ks = synth.batched_sbm(wl["n_graphs"], wl["graph_seed"])
    dev = torch.device("cuda")
    gs = [sf.csr_build(gr.n, torch.as_tensor(gr.src, device=dev), torch.as_tensor(gr.dst, device=dev), None)
          for gr in graphs]
    gos = [oracle_mod.csr_build(gr.n, gr.src, gr.dst, gr.w) for gr in graphs]
    # lam_hat from the oracle: 2 max_i s_i (the Gershgorin bound of the reading of §4.1 step 1)
    lams = [2.0 * float(oracle_mod.strength(go).max()) for go in gos]
    b = sf.batch_build(gs)
    n_tot, _, ng, offs = b.info()
    R = synth.gaussian_block(n_tot, eta, wl["r_seed"])
    coeffs = np.stack([oracle_mod.cheb_coeffs(lams[i], (0.05 + 0.1 * (i % 3)) * lams[i], p, True)[0]
                       for i in range(ng)])
    Y = sf.cheb_filter_batched(b, lams, coeffs, torch.as_tensor(R, dtype=torch.float32, device=dev),
                               sf.Opts(storage=sf.BF16))
    from helpers import dense_laplacian, dense_w, stored_block_error_model

    sizes = np.diff(offs)
    smallest = int(np.argmin(sizes))
    for i in (smallest, int(np.argmax(sizes)), 128):
        sl = slice(int(offs[i]), int(offs[i + 1]))
        Yo = oracle_mod.cheb_filter(gos[i], lams[i], coeffs[i], np.ascontiguousarray(R[sl][:, :2]))[0]
        if i == smallest:
            gr = graphs[i]
            lam = np.linalg.eigvalsh(dense_laplacian(dense_w(gr.n, gr.src, gr.dst)))
            # the GPU rounds R to BF16 as it packs it: the model includes that rounding
            bound = stored_block_error_model(2.0 * lam / lams[i] - 1.0, coeffs[i], 2.0 ** -8, "forward", True)
        else:
            bound = 5e-3
        for c in range(2):
            err = rel(Y[sl][:, c].cpu().numpy(), Yo[:, c])
            record_property(f"err_bf16_graph{i}_col{c}", err)
            record_property(f"bound_bf16_graph{i}", bound)
            assert err <= bound, (i, c, err, bound)
