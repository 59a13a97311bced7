"""GPU k-means (§4.1 step 6) against the oracle's Lloyd iterations on the same
FP32 rows and initial centroids.

Labels are integers decided by floating point; both sides decide them with
the FP32 fused-multiply-add sum in index order (ties to the lowest index), so
labels and the number of assignments must be equal. Centroids are means
rounded to FP32 on both sides, of sums taken differently (exact integer sums
of values rounded down to a fixed point far below FP32 resolution on the GPU, FP64
in row order in the oracle): equal up to one FP32 ulp. Inertia: FP64 sums in different orders,
1e-12 relative.
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


def mixture(n, d, k, seed, spread=1.0):
    rng = np.random.default_rng(seed)
    centres = rng.standard_normal((k, d)) * 2.0
    lab = rng.integers(0, k, n)
    F = (centres[lab] + spread * rng.standard_normal((n, d))).astype(np.float32)
    F /= np.linalg.norm(F, axis=1, keepdims=True)  # unit rows, like the features
    C0 = F[rng.choice(n, k, replace=False)].copy()
    return F, C0


def farthest_point_init(F, k, seed):
    """k rows: a random first one, then repeatedly the row farthest from those
    chosen (a deterministic k-means++ variant)."""
    rng = np.random.default_rng(seed)
    idx = [int(rng.integers(len(F)))]
    dmin = ((F - F[idx[0]]) ** 2).sum(1)
    for _ in range(k - 1):
        idx.append(int(np.argmax(dmin)))
        dmin = np.minimum(dmin, ((F - F[idx[-1]]) ** 2).sum(1))
    return F[idx].copy()


def check_same(sf, oracle_mod, F, C0, max_iter, mode):
    lo, Co, it_o, in_o = oracle_mod.kmeans(F, C0, max_iter)
    lab, C, it, inertia = sf.kmeans(torch.as_tensor(F, device="cuda"), torch.as_tensor(C0, device="cuda"),
                                    max_iter, mode)
    np.testing.assert_array_equal(lab.cpu().numpy(), lo)
    assert it == it_o
    Cg = C.cpu().numpy()
    ulp = np.abs(Cg.view(np.int32).astype(np.int64) - Co.view(np.int32).astype(np.int64))
    assert ulp.max() <= 1, ulp.max()
    assert inertia == pytest.approx(in_o, rel=1e-12)
    return lo, it_o


@pytest.mark.parametrize("d,k", [(32, 1), (32, 7), (64, 16), (128, 100), (128, 128), (96, 33)])
def test_kmeans_tensor_cores_match_oracle(sf, oracle_mod, d, k):
    # ragged row count: not a multiple of the 128-row tiles
    F, C0 = mixture(3001, d, k, seed=d + k)
    for mode in (sf.KMEANS_TENSOR, sf.KMEANS_TENSOR_SINGLE, sf.KMEANS_CUDA_CORES):
        check_same(sf, oracle_mod, F, C0, 12, mode)


def test_kmeans_iteration_limit_boundaries(sf, oracle_mod):
    """The host learns whether an assignment changed labels one assignment
    late; with max_iter just below, at and above the count at which labels
    stop changing, labels, centroids, inertia and the count still equal the
    oracle's (which stops after every assignment)."""
    F, C0 = mixture(2500, 64, 12, seed=21)
    _, _, it_free, _ = oracle_mod.kmeans(F, C0, 100)
    assert it_free >= 3
    for mode in (sf.KMEANS_TENSOR, sf.KMEANS_CUDA_CORES):
        for mi in (1, 2, it_free - 1, it_free, it_free + 1):
            check_same(sf, oracle_mod, F, C0, mi, mode)


def test_kmeans_other_shapes_use_cuda_cores(sf, oracle_mod):
    F, C0 = mixture(1500, 48, 200, seed=5)  # d not a multiple of 32, k > 128
    check_same(sf, oracle_mod, F, C0, 6, sf.KMEANS_AUTO)
    F, C0 = mixture(900, 30, 9, seed=6)  # d not a multiple of 4: scalar shared-memory loads
    check_same(sf, oracle_mod, F, C0, 6, sf.KMEANS_AUTO)
    F, C0 = mixture(700, 300, 5, seed=7)  # d > 256: a warp per row
    check_same(sf, oracle_mod, F, C0, 4, sf.KMEANS_AUTO)
    with pytest.raises(sf.SpecFiltError):
        sf.kmeans(torch.as_tensor(F, device="cuda"), torch.as_tensor(C0, device="cuda"), 3, sf.KMEANS_TENSOR)


def test_kmeans_cluster_tiles_and_scales(sf, oracle_mod):
    # k d too large for one tile of shared-memory sums (300 x 100 cells of 8 bytes): two cluster tiles
    F, C0 = mixture(2000, 300, 100, seed=8)
    check_same(sf, oracle_mod, F, C0, 4, sf.KMEANS_AUTO)
    # the fixed-point scale follows max |F_ij|: exact power-of-two rescalings far from unit rows
    F, C0 = mixture(2500, 64, 16, seed=9)
    for e in (40, -20):
        Fs, Cs = np.ldexp(F, e).astype(np.float32), np.ldexp(C0, e).astype(np.float32)
        for mode in (sf.KMEANS_TENSOR, sf.KMEANS_TENSOR_SINGLE, sf.KMEANS_CUDA_CORES):
            check_same(sf, oracle_mod, Fs, Cs, 8, mode)


def test_kmeans_structureless_rows_near_ties(sf, oracle_mod):
    # random unit rows and centroids: every row has several centroids at nearly the same distance, so the
    # tensor paths re-decide many rows; labels must still equal the FP32 decision of the oracle
    rng = np.random.default_rng(12)
    F = rng.standard_normal((20000, 128)).astype(np.float32)
    F /= np.linalg.norm(F, axis=1, keepdims=True)
    C0 = F[rng.choice(len(F), 100, replace=False)].copy()
    for mode in (sf.KMEANS_TENSOR, sf.KMEANS_TENSOR_SINGLE):
        check_same(sf, oracle_mod, F, C0, 4, mode)


def test_kmeans_ties_go_to_lowest_index(sf, oracle_mod):
    """Duplicated centroids tie exactly; the tensor-core gap is zero, so the
    rows go to the exact decision, which keeps the lower index."""
    F, C0 = mixture(2000, 64, 8, seed=7)
    C0 = np.concatenate([C0, C0[:3]], axis=0)  # centroids 8..10 duplicate 0..2
    lab, _ = check_same(sf, oracle_mod, F, C0, 1, sf.KMEANS_TENSOR)
    assert not np.isin(lab, [8, 9, 10]).any()


def test_kmeans_small_and_degenerate(sf, oracle_mod):
    F, C0 = mixture(5, 32, 3, seed=8)  # fewer rows than a tile
    check_same(sf, oracle_mod, F, C0, 5, sf.KMEANS_TENSOR)
    F, C0 = mixture(700, 32, 4, seed=9)
    C0[3] = 100.0  # far away: stays empty and keeps its coordinates
    check_same(sf, oracle_mod, F, C0, 4, sf.KMEANS_AUTO)
    F[17, 3] = np.nan
    with pytest.raises(sf.SpecFiltError):
        sf.kmeans(torch.as_tensor(F, device="cuda"), torch.as_tensor(C0, device="cuda"), 3)


def test_kmeans_on_filtered_features(sf, oracle_mod):
    """The path end to end on a small SBM: filter at the k-th eigenvalue,
    row-normalised features, k-means: the communities are recovered, and on
    the oracle's own features (cast to FP32) the GPU's labels equal the
    oracle's."""
    from paper_1509_08863_gb300 import synth

    n, k, eta, p = 1200, 6, 24, 60
    sizes = synth.community_sizes_equal(n, k)
    gr = synth.sbm_edges(n, sizes, 18.0, 0.02, seed=11)
    dev = torch.device("cuda")
    g = sf.csr_build(n, torch.as_tensor(gr.src, device=dev), torch.as_tensor(gr.dst, device=dev), None)
    _, lh = sf.lambda_max_estimate(g, 60, None, seed=3)
    R = torch.as_tensor(synth.gaussian_block(n, eta, 21), dtype=torch.float32, device=dev)
    mu = sf.cheb_moments(g, lh, R, p)
    lk = sf.dichotomy(mu, p, lh, k - 0.5)
    a = sf.cheb_coeffs(lh, lk, p, True)
    Y = sf.cheb_filter(g, lh, a, R)[0]
    Fe = sf.features(Y, True).cpu().numpy()
    C0 = farthest_point_init(Fe, k, seed=2)
    lab, _, _, _ = sf.kmeans(torch.as_tensor(Fe, device=dev), torch.as_tensor(C0, device=dev), 30)
    lab = lab.cpu().numpy()
    # purity of the communities the GPU path recovers (labels up to permutation)
    truth = gr.labels
    purity = sum(np.bincount(truth[lab == c]).max() for c in range(k) if (lab == c).any()) / n
    assert purity > 0.9, purity
    # labels equal the oracle's on the same FP32 features: the oracle's own (FP64 filter at its own
    # lam_hat and the cutoff between the k-th and (k+1)-th eigenvalues of the dense Laplacian)
    from helpers import dense_laplacian, dense_w, oracle_lambda_hat

    go = oracle_mod.csr_build(n, gr.src, gr.dst, gr.w)
    lam = np.linalg.eigvalsh(dense_laplacian(dense_w(n, gr.src, gr.dst)))
    lh_o = oracle_lambda_hat(oracle_mod, go, 60, seed=3)
    a_o = oracle_mod.cheb_coeffs(lh_o, 0.5 * (lam[k - 1] + lam[k]), p, True)
    Fo = oracle_mod.features(oracle_mod.cheb_filter(go, lh_o, a_o, synth.gaussian_block(n, eta, 21))[0], True)
    Fo32 = np.ascontiguousarray(Fo.astype(np.float32))
    check_same(sf, oracle_mod, Fo32, farthest_point_init(Fo32, k, seed=2), 30, sf.KMEANS_AUTO)
