// The stability measure of §4.3, Eq. (12), and the adjusted Rand index it is
// built on.
//
// gamma(k) for k in [kmin, kmax]: lam_k from the count's moments (one moment
// sweep of the probe block serves every k), then for each of the J
// realisations of the signals one forward sweep filters them at every lam_k
// at once (the multi-cutoff accumulation), the rows are normalised and
// k-means runs from `starts` seeded starts per k (lowest inertia kept);
// gamma(k) is the mean adjusted Rand index over the J (J - 1) / 2 pairs of
// realisations. The k-means starts pick rows with SplitMix64 (Steele, Lea,
// Flood, OOPSLA 2014) of the counter (j << 40) | (k << 20) | (t << 10) | c.
#include <math.h>

#include <vector>

#include "sf_internal.cuh"

namespace sf {

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

extern "C" SF_API sf_status sf_stability(const sf_graph *g, double lam_max, int32_t p, const float *Rc, const float *R,
                                         int32_t J, int32_t eta, int32_t kmin, int32_t kmax, int32_t max_iter,
                                         int32_t starts, uint64_t seed, const sf_opts *opts, void *stream,
                                         double *gamma, double *lam_k) {
    SF_ARG(g && Rc && R && gamma && lam_k, "null pointer");
    SF_ARG(J >= 2 && eta >= 1 && p >= 1, "need J >= 2, eta >= 1, p >= 1");
    SF_ARG(kmin >= 1 && kmax >= kmin && kmax <= 1023, "need 1 <= kmin <= kmax <= 1023");
    SF_ARG(max_iter >= 1 && starts >= 1 && starts <= 1023, "need max_iter >= 1 and 1 <= starts <= 1023");
    cudaStream_t s = (cudaStream_t)stream;
    const int32_t n = g->n;
    const int32_t K = kmax - kmin + 1;
    sf_opts o = {};
    if (opts) o = *opts;
    o.algo = SF_ALGO_FORWARD;  // every cutoff in one sweep
    sf_status st;
    // lam_k for every k from one moment sweep of the probes
    std::vector<double> mu((size_t)2 * p + 1), a((size_t)K * (p + 1));
    sf_opts om = o;
    if (om.storage == SF_F16) om.storage = SF_BF16;
    if ((st = sf_cheb_moments(g, lam_max, Rc, SF_F32, eta, p, mu.data(), &om, stream))) return st;
    for (int32_t q = 0; q < K; ++q) {
        if ((st = sf_dichotomy(mu.data(), p, lam_max, (double)(kmin + q) - 0.5, 1, 40, 1e-9, &lam_k[q]))) return st;
        if ((st = sf_cheb_coeffs(lam_max, &lam_k[q], 1, p, 1, a.data() + (size_t)q * (p + 1)))) return st;
    }
    const int64_t blk = (int64_t)n * eta;
    Scratch sc(s);
    float *Y = nullptr, *C0 = nullptr;
    int32_t *labels = nullptr, *trial = nullptr, *rows = nullptr;
    if ((st = sc.get(&Y, (size_t)K * blk)) || (st = sc.get(&C0, (size_t)kmax * eta)) ||
        (st = sc.get(&labels, (size_t)J * K * n)) || (st = sc.get(&trial, (size_t)n)) ||
        (st = sc.get(&rows, (size_t)kmax)))
        return st;
    std::vector<int32_t> hrows((size_t)kmax);
    for (int32_t j = 0; j < J; ++j) {
        if ((st = sf_cheb_filter(g, lam_max, a.data(), K, p, R + (size_t)j * blk, SF_F32, eta, Y, &o, stream)))
            return st;
        for (int32_t q = 0; q < K; ++q) {
            const int32_t k = kmin + q;
            float *Fq = Y + (size_t)q * blk;
            if ((st = sf_features(Fq, n, eta, 1, Fq, stream))) return st;
            double best = INFINITY;
            for (int32_t t = 0; t < starts; ++t) {
                for (int32_t c = 0; c < k; ++c) {
                    const uint64_t ctr = ((uint64_t)j << 40) | ((uint64_t)k << 20) | ((uint64_t)t << 10) | (uint64_t)c;
                    hrows[c] = (int32_t)(splitmix64_at(seed, ctr) % (uint64_t)n);
                }
                SF_CHECK_CUDA(cudaMemcpyAsync(rows, hrows.data(), sizeof(int32_t) * k, cudaMemcpyHostToDevice, s));
                gather_rows_kernel<<<sm_count(), 256, 0, s>>>(Fq, eta, rows, k, C0);
                if ((st = check_launch("gather_rows_kernel"))) return st;
                int32_t it = 0;
                double inertia = 0.0;
                if ((st = sf_kmeans(Fq, n, eta, k, C0, max_iter, SF_KMEANS_AUTO, trial, &it, &inertia, stream)))
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
