// The stability measure of §4.3, Eq. (12), and the adjusted Rand index it is
// built on.
//
// gamma(k) for k in [kmin, kmax]: lam_k from the count's moments (one moment
// sweep of the probe block serves every k); the J realisations of the signals,
// placed side by side as one block of J * eta columns, are filtered at every
// lam_k in one forward sweep (the multi-cutoff accumulation; the columns are
// independent), each realisation's rows are normalised and k-means runs from
// `starts` seeded starts per k (lowest inertia kept); gamma(k) is the mean
// adjusted Rand index over the J (J - 1) / 2 pairs of realisations. The
// k-means starts pick rows with SplitMix64 (Steele, Lea, Flood, OOPSLA 2014)
// of the counter (j << 40) | (k << 20) | (t << 10) | c. The filter order can
// be chosen so that the filters at adjacent k differ (resolving_order).
#include <math.h>

#include <vector>

#include "sf_internal.cuh"

namespace sf {

constexpr int32_t kStabilityOrderCap = 20000;  // the automatic filter order stops here

__global__ void contingency_kernel(const int32_t *a, const int32_t *b, int32_t n, int32_t ka, int32_t kb,
                                   unsigned long long *t, int32_t *bad) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = a[i], v = b[i];
        if (u < 0 || u >= ka || v < 0 || v >= kb) {
            *bad = 1;
            continue;
        }
        atomicAdd(t + (int64_t)u * kb + v, 1ull);
    }
}

__global__ void gather_rows_kernel(const float *F, int32_t d, const int32_t *rows, int32_t k, float *C) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)k * d;
         t += (int64_t)gridDim.x * blockDim.x)
        C[t] = F[(int64_t)rows[t / d] * d + t % d];
}

// R_all[i][j * eta + c] = R[j][i][c]: the J realisations side by side as one block
__global__ void interleave_realisations_kernel(const float *R, int32_t J, int32_t n, int32_t eta, float *R_all) {
    const int64_t total = (int64_t)J * n * eta;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = t / ((int64_t)n * eta);
        const int64_t r = t - j * n * eta;
        const int64_t i = r / eta, c = r - i * eta;
        R_all[i * ((int64_t)J * eta) + j * eta + c] = R[t];
    }
}

// F[i][c] = Y[i][off + c] / ||Y[i][off .. off + w)||: the row-normalised features of one
// realisation's columns (the same per-lane FP32 partials and FP64 sum as sf_features)
__global__ void __launch_bounds__(256) segment_features_kernel(const float *Y, int32_t n, int32_t ld, int32_t off,
                                                               int32_t w, float *F) {
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp0; i < n; i += nw) {
        const float *y = Y + i * ld + off;
        float *f = F + i * w;
        float part = 0.f;
        for (int c = lane; c < w; c += 32) part = fmaf(y[c], y[c], part);
        double ss = (double)part;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        const double nrm = sqrt(ss);
        const float inv = nrm > 0.0 ? (float)(1.0 / nrm) : 0.0f;
        for (int c = lane; c < w; c += 32) f[c] = y[c] * inv;
    }
}

// The filter order at which adjacent cutoffs give different filters: in
// theta = arccos(2 lambda / lam_max - 1) a Jackson-damped series of order p
// has a transition of standard deviation about pi / (p + 2) around its
// cutoff, so +-2 of them fit between two cutoffs once
// p + 2 >= 4 pi / (their theta gap). lam holds ascending cutoffs.
static int32_t resolving_order(const std::vector<double> &lam, double lam_max, int32_t p_min, int32_t p_cap) {
    double gap = INFINITY;
    for (size_t q = 1; q < lam.size(); ++q) {
        const double t0 = acos(fmin(1.0, fmax(-1.0, 2.0 * lam[q - 1] / lam_max - 1.0)));
        const double t1 = acos(fmin(1.0, fmax(-1.0, 2.0 * lam[q] / lam_max - 1.0)));
        gap = fmin(gap, fabs(t0 - t1));
    }
    if (!(gap > 0.0)) return p_cap;
    const double want = ceil(4.0 * M_PI / gap) - 2.0;
    if (want >= (double)p_cap) return p_cap;
    return want > (double)p_min ? (int32_t)want : p_min;
}

static uint64_t splitmix64_at(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace sf

using namespace sf;

extern "C" SF_API sf_status sf_adjusted_rand(const int32_t *a, const int32_t *b, int32_t n, int32_t ka, int32_t kb,
                                             void *stream, double *ari) {
    SF_ARG(a && b && ari, "a/b/ari is NULL");
    SF_ARG(n >= 1 && ka >= 1 && kb >= 1, "need n, ka, kb >= 1");
    SF_ARG((int64_t)ka * kb <= (1ll << 24), "ka * kb must be <= 2^24");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t cells = (int64_t)ka * kb;
    Scratch sc(s);
    unsigned long long *t = nullptr;
    int32_t *bad = nullptr;
    sf_status st;
    if ((st = sc.get(&t, (size_t)cells)) || (st = sc.get(&bad, 1))) return st;
    SF_CHECK_CUDA(cudaMemsetAsync(t, 0, sizeof(unsigned long long) * (size_t)cells, s));
    SF_CHECK_CUDA(cudaMemsetAsync(bad, 0, sizeof(int32_t), s));
    contingency_kernel<<<4 * sm_count(), 256, 0, s>>>(a, b, n, ka, kb, t, bad);
    if ((st = check_launch("contingency_kernel"))) return st;
    std::vector<unsigned long long> h((size_t)cells);
    int32_t hbad = 0;
    SF_CHECK_CUDA(cudaMemcpyAsync(h.data(), t, sizeof(unsigned long long) * (size_t)cells, cudaMemcpyDeviceToHost, s));
    SF_CHECK_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    SF_CHECK_CUDA(cudaStreamSynchronize(s));
    SF_ARG(!hbad, "a label lies outside [0, ka) or [0, kb)");
    // Hubert and Arabie (1985): pair counts x (x - 1) / 2 of the cells and the margins
    std::vector<double> ra((size_t)ka, 0.0), rb((size_t)kb, 0.0);
    double sij = 0.0;
    for (int64_t u = 0; u < cells; ++u) {
        const double x = (double)h[u];
        sij += 0.5 * x * (x - 1.0);
        ra[u / kb] += x;
        rb[u % kb] += x;
    }
    double sa = 0.0, sb = 0.0;
    for (int32_t u = 0; u < ka; ++u) sa += 0.5 * ra[u] * (ra[u] - 1.0);
    for (int32_t v = 0; v < kb; ++v) sb += 0.5 * rb[v] * (rb[v] - 1.0);
    const double pairs = 0.5 * (double)n * (double)(n - 1);
    const double expct = pairs > 0.0 ? sa * sb / pairs : 0.0;
    const double top = 0.5 * (sa + sb);
    *ari = (top == expct) ? 1.0 : (sij - expct) / (top - expct);
    return SF_OK;
}

extern "C" SF_API sf_status sf_stability(const sf_graph *g, double lam_max, int32_t p, int32_t p_filter,
                                         const float *Rc, const float *R, int32_t J, int32_t eta, int32_t kmin,
                                         int32_t kmax, int32_t max_iter, int32_t starts, uint64_t seed,
                                         const sf_opts *opts, void *stream, double *gamma, double *lam_k,
                                         int32_t *p_used) {
    SF_ARG(g && Rc && R && gamma && lam_k, "null pointer");
    SF_ARG(J >= 2 && eta >= 1 && p >= 1, "need J >= 2, eta >= 1, p >= 1");
    SF_ARG(p_filter >= 0 && p_filter <= kStabilityOrderCap, "p_filter must be in [0, %d] (0: automatic)",
           kStabilityOrderCap);
    SF_ARG((int64_t)J * eta <= (1 << 20), "J * eta must be <= 2^20");
    SF_ARG(kmin >= 1 && kmax >= kmin && kmax <= 1023, "need 1 <= kmin <= kmax <= 1023");
    SF_ARG(max_iter >= 1 && starts >= 1 && starts <= 1023, "need max_iter >= 1 and 1 <= starts <= 1023");
    cudaStream_t s = (cudaStream_t)stream;
    const int32_t n = g->n;
    const int32_t K = kmax - kmin + 1;
    sf_opts o = {};
    if (opts) o = *opts;
    o.algo = SF_ALGO_FORWARD;  // every cutoff in one sweep
    sf_status st;
    sf_opts om = o;
    if (om.storage == SF_F16) om.storage = SF_BF16;
    // lam_k for every k (and the neighbours kmin - 1, kmax + 1 that bound the gaps) from one
    // moment sweep of the probes at order pc
    const int32_t klo = kmin > 1 ? kmin - 1 : kmin, khi = kmax + 1;
    std::vector<double> lam_all((size_t)(khi - klo + 1));
    auto estimate = [&](int32_t pc) -> sf_status {  // moments at order pc, the dichotomy for each k
        std::vector<double> mu((size_t)2 * pc + 1);
        sf_status e = sf_cheb_moments(g, lam_max, Rc, SF_F32, eta, pc, mu.data(), &om, stream);
        if (e) return e;
        for (int32_t k = klo; k <= khi; ++k)
            if ((e = sf_dichotomy(mu.data(), pc, lam_max, (double)k - 0.5, 1, 40, 1e-9, &lam_all[k - klo])))
                return e;
        return SF_OK;
    };
    if ((st = estimate(p))) return st;
    // automatic order: resolve the gaps between the estimated cutoffs (the count keeps its order p:
    // its FP32 moments of degree up to 2p lose accuracy at the orders the filters may need)
    const int32_t pf = p_filter > 0 ? p_filter : resolving_order(lam_all, lam_max, p, kStabilityOrderCap);
    if (p_used) *p_used = pf;
    std::vector<double> a((size_t)K * (pf + 1));
    for (int32_t q = 0; q < K; ++q) {
        lam_k[q] = lam_all[kmin + q - klo];
        if ((st = sf_cheb_coeffs(lam_max, &lam_k[q], 1, pf, 1, a.data() + (size_t)q * (pf + 1)))) return st;
    }
    // the J realisations side by side: one block of J * eta independent columns, filtered at every
    // lam_k in one multi-cutoff forward sweep (§3.1: the columns are independent signals)
    const int32_t W = J * eta;
    const int64_t blk = (int64_t)n * W;
    Scratch sc(s);
    float *Rall = nullptr, *Y = nullptr, *F = nullptr, *C0 = nullptr;
    int32_t *labels = nullptr, *trial = nullptr, *rows = nullptr;
    if ((st = sc.get(&Rall, (size_t)blk)) || (st = sc.get(&Y, (size_t)K * blk)) ||
        (st = sc.get(&F, (size_t)n * eta)) || (st = sc.get(&C0, (size_t)kmax * eta)) ||
        (st = sc.get(&labels, (size_t)J * K * n)) || (st = sc.get(&trial, (size_t)n)) ||
        (st = sc.get(&rows, (size_t)kmax)))
        return st;
    if (blk > 0) {
        interleave_realisations_kernel<<<4 * sm_count(), 256, 0, s>>>(R, J, n, eta, Rall);
        if ((st = check_launch("interleave_realisations_kernel"))) return st;
    }
    if ((st = sf_cheb_filter(g, lam_max, a.data(), K, pf, Rall, SF_F32, W, Y, &o, stream))) return st;
    std::vector<int32_t> hrows((size_t)kmax);
    for (int32_t j = 0; j < J; ++j) {
        for (int32_t q = 0; q < K; ++q) {
            const int32_t k = kmin + q;
            segment_features_kernel<<<2 * sm_count(), 256, 0, s>>>(Y + (size_t)q * blk, n, W, j * eta, eta, F);
            if ((st = check_launch("segment_features_kernel"))) return st;
            double best = INFINITY;
            for (int32_t t = 0; t < starts; ++t) {
                for (int32_t c = 0; c < k; ++c) {
                    const uint64_t ctr = ((uint64_t)j << 40) | ((uint64_t)k << 20) | ((uint64_t)t << 10) | (uint64_t)c;
                    hrows[c] = (int32_t)(splitmix64_at(seed, ctr) % (uint64_t)n);
                }
                SF_CHECK_CUDA(cudaMemcpyAsync(rows, hrows.data(), sizeof(int32_t) * k, cudaMemcpyHostToDevice, s));
                gather_rows_kernel<<<sm_count(), 256, 0, s>>>(F, eta, rows, k, C0);
                if ((st = check_launch("gather_rows_kernel"))) return st;
                int32_t it = 0;
                double inertia = 0.0;
                if ((st = sf_kmeans(F, n, eta, k, C0, max_iter, SF_KMEANS_AUTO, trial, &it, &inertia, stream)))
                    return st;
                if (inertia < best) {
                    best = inertia;
                    SF_CHECK_CUDA(cudaMemcpyAsync(labels + ((size_t)j * K + q) * n, trial, sizeof(int32_t) * n,
                                                  cudaMemcpyDeviceToDevice, s));
                }
            }
        }
    }
    for (int32_t q = 0; q < K; ++q) {
        const int32_t k = kmin + q;
        double acc = 0.0;
        int64_t pairs = 0;
        for (int32_t i = 0; i < J; ++i)
            for (int32_t j = i + 1; j < J; ++j) {
                double ari = 0.0;
                if ((st = sf_adjusted_rand(labels + ((size_t)i * K + q) * n, labels + ((size_t)j * K + q) * n, n, k, k,
                                           stream, &ari)))
                    return st;
                acc += ari;
                ++pairs;
            }
        gamma[q] = acc / (double)pairs;
    }
    return SF_OK;
}
