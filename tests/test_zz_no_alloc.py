"""The allocation-free moment sweep (sf_cheb_moments_noalloc).

It is meant for callers that cannot allocate device memory when they need
the moments (stream capture, a framework-owned allocator, latency-bound
loops): all of its working memory comes from one fixed array compiled into
the library. These tests call it through the C ABI and check it against the
allocating entry point, sf_cheb_moments, twice in a row -- the array keeps
the previous call's contents, so a missing reset would show up on the second
call. This file is collected last so that a failure here cannot hide the
results of the other tests.
"""
import ctypes as C

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


def _graph(sf, n, k, deg, seed):
    from paper_1509_08863_gb300 import synth

    gr = synth.sbm_edges(n, synth.community_sizes_equal(n, k), deg, 0.1, seed=seed)
    dev = torch.device("cuda")
    return sf.csr_build(n, torch.as_tensor(gr.src, device=dev), torch.as_tensor(gr.dst, device=dev), None)


def _noalloc(sf, g, lam, R, p):
    mu = np.zeros(2 * p + 1)
    L = sf.lib()
    st = L.sf_cheb_moments_noalloc(g.handle, float(lam), C.c_void_p(R.data_ptr()), R.shape[1], p,
                                   mu.ctypes.data_as(C.POINTER(C.c_double)),
                                   C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, mu


@pytest.mark.parametrize("n,n_sig,p", [(3001, 24, 40), (20000, 64, 25)])
def test_noalloc_moments_match_allocating_entry(sf, n, n_sig, p):
    g = _graph(sf, n, 8, 12.0, seed=n)
    _, lam = sf.lambda_max_estimate(g, 40, None, seed=3)
    R = torch.randn(n, n_sig, device="cuda") / np.sqrt(n_sig)
    ref = sf.cheb_moments(g, lam, R, p)  # also builds the graph's sweep layout
    tol = np.array([2e-6 * (m + 1) * ref[0] for m in range(2 * p + 1)])
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


def test_noalloc_rejects_oversize_and_unprepared(sf):
    g = _graph(sf, 400_000, 4, 4.0, seed=5)
    R = torch.randn(400_000, 16, device="cuda")
    st, _ = _noalloc(sf, g, 20.0, R, 3)
    assert st == 1 and b"sweep layout" in sf.lib().sf_last_error()  # no layout yet
    sf.cheb_moments(g, 20.0, R, 3)
    st, _ = _noalloc(sf, g, 20.0, R, 3)
    assert st == 1 and b"working memory" in sf.lib().sf_last_error()
