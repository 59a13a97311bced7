"""The allocation-free moment sweep (sf_cheb_moments_noalloc).

It is meant for callers that cannot allocate device memory when they need
the moments -- a framework whose own caching allocator owns the device
memory, or a latency-bound loop that cannot afford an allocator call: all of
its working memory comes from one fixed array compiled into the library.
These tests call it through the C ABI and check it against the allocating
entry point, sf_cheb_moments, twice in a row -- the array keeps the previous
call's contents, so a missing reset would show up on the second call -- and
once against the FP64 oracle. The two entry points reduce the FP64 dot
products in the same kernels but may cut the block into different slabs, so
they agree within the FP64 reduction-order tolerance of the moment tests,
2e-6 (m + 1) mu_0. This file is collected last so that a failure here cannot
hide the results of the other tests.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

SF_ERR_ARG, SF_ERR_NUMERIC = 1, 5


@pytest.fixture(scope="module")
def sf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_08863_gb300 import build

    build.build()
    import paper_1509_08863_gb300 as m

    return m


def _edges(n, k, deg, seed):
    from paper_1509_08863_gb300 import synth

    return synth.sbm_edges(n, synth.community_sizes_equal(n, k), deg, 0.1, seed=seed)


def _graph(sf, gr, n):
    dev = torch.device("cuda")
    return sf.csr_build(n, torch.as_tensor(gr.src, device=dev), torch.as_tensor(gr.dst, device=dev), None)


def _noalloc(sf, g, lam, R, p):
    mu = np.zeros(2 * p + 1)
    L = sf.lib()
    st = L.sf_cheb_moments_noalloc(g.handle, float(lam), C.c_void_p(R.data_ptr()), R.shape[1], p,
                                   mu.ctypes.data_as(C.POINTER(C.c_double)),
                                   C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, mu


def _tol(mu0, p):
    return np.array([2e-6 * (m + 1) * mu0 for m in range(2 * p + 1)])


# (60000, 128) once needed more than the array at the default slab width; (300000, 32)
# fits only with 16-column slabs, so the call runs two slabs
@pytest.mark.parametrize("n,n_sig,p", [(3001, 24, 40), (20000, 64, 25), (60000, 128, 10), (300000, 32, 6)])
def test_noalloc_moments_match_allocating_entry(sf, n, n_sig, p):
    g = _graph(sf, _edges(n, 8, 12.0, seed=n), n)
    _, lam = sf.lambda_max_estimate(g, 40, None, seed=3)
    R = torch.randn(n, n_sig, device="cuda") / np.sqrt(n_sig)
    ref = sf.cheb_moments(g, lam, R, p)  # also builds the graph's sweep layout
    tol = _tol(ref[0], p)
    first = None
    for call in range(2):
        st, mu = _noalloc(sf, g, lam, R, p)
        assert st == 0, sf.lib().sf_last_error()
        assert np.all(np.abs(mu - ref) <= tol), (call, np.abs(mu - ref).max())
        if first is None:
            first = mu
        else:
            np.testing.assert_array_equal(mu, first)
    # different sizes and orders after a larger call: stale contents must not leak in
    R2 = torch.randn(n, 8, device="cuda")
    ref2 = sf.cheb_moments(g, lam, R2, 7)
    st, mu2 = _noalloc(sf, g, lam, R2, 7)
    assert st == 0
    assert np.all(np.abs(mu2 - ref2) <= 2e-6 * 16 * ref2[0])


def test_noalloc_moments_match_oracle(sf):
    import oracle
    from paper_1509_08863_gb300 import synth

    oracle.build()
    n, n_sig, p = 2000, 24, 30
    gr = _edges(n, 8, 12.0, seed=7)
    g = _graph(sf, gr, n)
    go = oracle.csr_build(n, gr.src, gr.dst, gr.w)
    _, lam = sf.lambda_max_estimate(g, 50, None, seed=1)
    R = synth.gaussian_block(n, n_sig, seed=9)
    Rt = torch.as_tensor(R, dtype=torch.float32, device="cuda")
    sf.cheb_moments(g, lam, Rt, 2)  # builds the sweep layout
    st, mu = _noalloc(sf, g, lam, Rt, p)
    assert st == 0, sf.lib().sf_last_error()
    muo = oracle.moments(go, lam, R, 2 * p)
    assert np.all(np.abs(mu - muo) <= _tol(muo[0], p)), np.abs(mu - muo).max()


def test_noalloc_allocates_nothing(sf):
    n, n_sig, p = 50000, 32, 12
    g = _graph(sf, _edges(n, 8, 12.0, seed=11), n)
    R = torch.randn(n, n_sig, device="cuda")
    _, lam = sf.lambda_max_estimate(g, 40, None, seed=3)
    sf.cheb_moments(g, lam, R, 2)
    st, _ = _noalloc(sf, g, lam, R, p)  # the first call on the device looks the array up
    assert st == 0
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        st, _ = _noalloc(sf, g, lam, R, p)
        assert st == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


def test_noalloc_numeric_checks(sf):
    # lam_max below the spectrum makes ||T_j R|| grow: SF_ERR_NUMERIC, as from sf_cheb_moments
    n = 5000
    g = _graph(sf, _edges(n, 8, 12.0, seed=13), n)
    _, lam = sf.lambda_max_estimate(g, 40, None, seed=3)
    R = torch.randn(n, 16, device="cuda")
    sf.cheb_moments(g, lam, R, 2)
    st, _ = _noalloc(sf, g, 0.5 * lam, R, 12)
    assert st == SF_ERR_NUMERIC and b"below" in sf.lib().sf_last_error()
    Rn = R.clone()
    Rn[17, 3] = float("nan")
    st, _ = _noalloc(sf, g, lam, Rn, 4)
    assert st == SF_ERR_NUMERIC and b"non-finite" in sf.lib().sf_last_error()
    st, mu = _noalloc(sf, g, lam, R, 4)  # the next call works
    assert st == 0 and np.all(np.isfinite(mu))


def test_noalloc_rejects_oversize_and_unprepared(sf):
    # 800,000 rows need 3 blocks of >= 8 FP32 columns, about 77 MB: more than the 64 MiB array
    n = 800_000
    g = _graph(sf, _edges(n, 4, 4.0, seed=5), n)
    R = torch.randn(n, 16, device="cuda")
    st, _ = _noalloc(sf, g, 20.0, R, 3)
    assert st == SF_ERR_ARG and b"sweep layout" in sf.lib().sf_last_error()  # no layout yet
    _, lam = sf.lambda_max_estimate(g, 20, None, seed=3)  # builds the layout
    sf.cheb_moments(g, lam, R, 3)
    st, _ = _noalloc(sf, g, lam, R, 3)
    assert st == SF_ERR_ARG and b"working memory" in sf.lib().sf_last_error()
