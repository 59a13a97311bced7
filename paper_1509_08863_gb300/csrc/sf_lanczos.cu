// lambda_N estimate (§4.1 step 1) by Lanczos in FP64 on the device, and the
// feature rows of Eq. (6) / Eq. (11) (optionally L2-normalised).
#include <math.h>

#include "sf_internal.cuh"

namespace sf {

// SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014): state += golden gamma, then two xor-shift-multiply
// rounds. Maps (seed, i) to a uniform double in [-1, 1).
__device__ __forceinline__ double splitmix_uniform(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

__global__ void lanczos_init_kernel(double *v, const double *v0, uint64_t seed, int32_t n) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = v0 ? v0[i] : splitmix_uniform(seed, (uint64_t)i);
}

// part[b] = block partial of sum x_i y_i (fixed strided order per block).
template <int BS>
__device__ void block_dot_store(double acc, double *part) {
    __shared__ double sh[BS];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = BS / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// w = L v over the sliced-ELL copy: one thread per row, indices read four at a
// time and eight gathers in flight; partial <w, v>. Padding entries gather
// v[n] = 0. The row sum runs in entry order (the CSR column order).
__global__ void __launch_bounds__(256) lap_spmv_sell_kernel(int32_t n, const int32_t *sptr, const int32_t *perm,
                                                            const int32_t *idx, const float *sval,
                                                            const double *strength, const double *v, double *w,
                                                            double *part) {
    double dot = 0.0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = perm[t];
        if (i < 0) continue;
        const int32_t sl = (int32_t)(t / kSliceRows), pos = (int32_t)(t % kSliceRows);
        const int32_t so = sptr[sl], ls = (sptr[sl + 1] - so) / kSliceRows;
        const int64_t eo = (int64_t)so + (int64_t)pos * ls;
        double acc = 0.0;
        int32_t e = 0;
        for (; e + 8 <= ls; e += 8) {  // eight gathers in flight
            const int4 ka = __ldg(reinterpret_cast<const int4 *>(idx + eo + e));
            const int4 kb = __ldg(reinterpret_cast<const int4 *>(idx + eo + e + 4));
            const int32_t k[8] = {ka.x, ka.y, ka.z, ka.w, kb.x, kb.y, kb.z, kb.w};
            double x[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) x[u] = __ldg(v + k[u]);
            if (sval) {
                const float4 ca = __ldg(reinterpret_cast<const float4 *>(sval + eo + e));
                const float4 cb = __ldg(reinterpret_cast<const float4 *>(sval + eo + e + 4));
                const float c[8] = {ca.x, ca.y, ca.z, ca.w, cb.x, cb.y, cb.z, cb.w};
#pragma unroll
                for (int u = 0; u < 8; ++u) acc += (double)c[u] * x[u];
            } else {
#pragma unroll
                for (int u = 0; u < 8; ++u) acc += x[u];
            }
        }
        if (e < ls) {  // ls is a multiple of 4
            const int4 k = __ldg(reinterpret_cast<const int4 *>(idx + eo + e));
            const double x0 = __ldg(v + k.x), x1 = __ldg(v + k.y), x2 = __ldg(v + k.z), x3 = __ldg(v + k.w);
            if (sval) {
                const float4 c = __ldg(reinterpret_cast<const float4 *>(sval + eo + e));
                acc += (double)c.x * x0;
                acc += (double)c.y * x1;
                acc += (double)c.z * x2;
                acc += (double)c.w * x3;
            } else {
                acc += x0;
                acc += x1;
                acc += x2;
                acc += x3;
            }
        }
        const double vi = v[i];
        const double wi = strength[i] * vi - acc;
        w[i] = wi;
        dot += wi * vi;
    }
    block_dot_store<256>(dot, part);
}

// w -= alpha[k] v + beta[k] vp; partial |w|^2.
__global__ void lanczos_update_kernel(int32_t n, double *w, const double *v, const double *vp, const double *alpha,
                                      const double *beta, int k, double *part) {
    const double a = alpha[k], b = (k > 0) ? beta[k - 1] : 0.0;
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double x = w[i] - a * v[i] - (k > 0 ? b * vp[i] : 0.0);
        w[i] = x;
        acc += x * x;
    }
    block_dot_store<256>(acc, part);
}

// out[k] = scale-function of the sum of part[0..count)
__global__ void lanczos_scalar_kernel(const double *part, int count, double *out, int k, int do_sqrt) {
    __shared__ double sh[256];
    double acc = 0.0;
    for (int t = threadIdx.x; t < count; t += blockDim.x) acc += part[t];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[k] = do_sqrt ? sqrt(sh[0]) : sh[0];
}

__global__ void lanczos_scale_kernel(int32_t n, const double *w, const double *nrm, int k, double *v) {
    const double inv = 1.0 / nrm[k];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = w[i] * inv;
}

__global__ void sumsq_kernel(int32_t n, const double *v, double *part) {
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc += v[i] * v[i];
    block_dot_store<256>(acc, part);
}

// ------------------------------------------------------------ features
// One warp per row, in FP32: the row is first scaled by the power of two that
// brings its largest magnitude into [1/2, 1) (exact), so that the sum of
// squares neither underflows nor overflows; F = y * (scale / sqrt(sum)).
// Rows of zero norm are written as zeros (rows with an infinite or NaN entry
// as y * 0).
__global__ void __launch_bounds__(256) features_kernel(const float *Y, int32_t n, int32_t n_sig, int32_t normalize,
                                                       float *F) {
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp0; i < n; i += nw) {
        const float *y = Y + i * n_sig;
        float *f = F + i * n_sig;
        if (!normalize) {
            for (int c = lane; c < n_sig; c += 32) f[c] = y[c];
            continue;
        }
        float m = 0.f;
        for (int c = lane; c < n_sig; c += 32) m = fmaxf(m, fabsf(y[c]));
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
        float inv = 0.f;
        if (m > 0.f && m <= 3.4028235e38f) {
            int e;
            frexpf(m, &e);                                        // m = fr * 2^e, fr in [1/2, 1)
            const float sc = ldexpf(1.0f, e < -125 ? 125 : -e);  // exact power of two
            float ss = 0.f;
            for (int c = lane; c < n_sig; c += 32) {
                const float v = y[c] * sc;
                ss = fmaf(v, v, ss);
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, off);
            if (ss > 0.f && ss <= 3.4028235e38f) inv = sc / sqrtf(ss);
        }
        for (int c = lane; c < n_sig; c += 32) f[c] = y[c] * inv;
    }
}

// Row sums of squares (FP64 per row from per-lane FP32 partials), one warp per row.
__global__ void __launch_bounds__(256) row_sumsq_kernel(const float *Y, int32_t n, int32_t n_sig, double *out) {
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp0; i < n; i += nw) {
        const float *y = Y + i * n_sig;
        float part = 0.f;
        for (int c = lane; c < n_sig; c += 32) part = fmaf(y[c], y[c], part);
        double ss = (double)part;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, off);
        if (lane == 0) out[i] = ss;
    }
}

// F = Y / sqrt(sumsq) row by row (rows with sumsq == 0 become zero).
__global__ void __launch_bounds__(256) row_scale_kernel(const float *Y, int32_t n, int32_t n_sig, const double *sumsq,
                                                        float *F) {
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp0; i < n; i += nw) {
        const double ss = sumsq[i];
        const float inv = ss > 0.0 ? (float)(1.0 / sqrt(ss)) : 0.0f;
        for (int c = lane; c < n_sig; c += 32) F[i * n_sig + c] = Y[i * n_sig + c] * inv;
    }
}

}  // namespace sf

using namespace sf;

extern "C" {

SF_API sf_status sf_row_sumsq(const float *Y, int32_t n, int32_t n_sig, double *sumsq, void *stream) {
    SF_ARG(Y && sumsq, "Y/sumsq is NULL");
    SF_ARG(n >= 0 && n_sig >= 1, "need n >= 0 and n_sig >= 1");
    if (n == 0) return SF_OK;
    int64_t grid = ((int64_t)n * 32 + 255) / 256;
    const int64_t cap = (int64_t)sm_count() * 8;
    if (grid > cap) grid = cap;
    row_sumsq_kernel<<<(unsigned)grid, 256, 0, (cudaStream_t)stream>>>(Y, n, n_sig, sumsq);
    return check_launch("row_sumsq_kernel");
}

SF_API sf_status sf_features_scaled(const float *Y, int32_t n, int32_t n_sig, const double *sumsq, float *F,
                                    void *stream) {
    SF_ARG(Y && sumsq && F, "Y/sumsq/F is NULL");
    SF_ARG(n >= 0 && n_sig >= 1, "need n >= 0 and n_sig >= 1");
    if (n == 0) return SF_OK;
    int64_t grid = ((int64_t)n * 32 + 255) / 256;
    const int64_t cap = (int64_t)sm_count() * 8;
    if (grid > cap) grid = cap;
    row_scale_kernel<<<(unsigned)grid, 256, 0, (cudaStream_t)stream>>>(Y, n, n_sig, sumsq, F);
    return check_launch("row_scale_kernel");
}

SF_API sf_status sf_lambda_max_estimate(const sf_graph *g, int32_t iters, const double *v0, uint64_t seed,
                                        void *stream, double *theta_max, double *lam_hat) {
    SF_ARG(g, "graph is NULL");
    SF_ARG(iters >= 1 && iters <= 10000, "iters must be in [1, 10000]");
    SF_ARG(g->device == current_device(), "graph lives on another device");
    cudaStream_t s = (cudaStream_t)stream;
    const int32_t n = g->n;
    if (iters > n) iters = n;
    Scratch sc(s);
    double *v = nullptr, *vp = nullptr, *w = nullptr, *part = nullptr, *alpha = nullptr, *beta = nullptr,
           *nrm = nullptr;
    sf_status st;
    const int grid = 4 * sm_count();
    // one extra element, kept 0: the padding entries of the sliced-ELL copy gather v[n]
    if ((st = sc.get(&v, (size_t)n + 1)) || (st = sc.get(&vp, (size_t)n + 1)) || (st = sc.get(&w, (size_t)n + 1)) ||
        (st = sc.get(&part, grid)) || (st = sc.get(&alpha, iters)) || (st = sc.get(&beta, iters)) ||
        (st = sc.get(&nrm, 1)))
        return st;
    SF_CHECK_CUDA(cudaMemsetAsync(v, 0, sizeof(double) * ((size_t)n + 1), s));
    SF_CHECK_CUDA(cudaMemsetAsync(vp, 0, sizeof(double) * ((size_t)n + 1), s));
    SF_CHECK_CUDA(cudaMemsetAsync(w, 0, sizeof(double) * ((size_t)n + 1), s));
    {
        std::lock_guard<std::mutex> lk(g->sell_mu);
        if ((st = sell_build(&g->sell, g->n, g->rowptr, g->colidx, g->unit_weights ? nullptr : g->val, s))) return st;
    }
    const SellMatrix &S = g->sell;
    lanczos_init_kernel<<<(n + 255) / 256, 256, 0, s>>>(w, v0, seed, n);
    if ((st = check_launch("lanczos_init_kernel"))) return st;
    sumsq_kernel<<<grid, 256, 0, s>>>(n, w, part);
    if ((st = check_launch("sumsq_kernel"))) return st;
    lanczos_scalar_kernel<<<1, 256, 0, s>>>(part, grid, nrm, 0, 1);
    if ((st = check_launch("lanczos_scalar_kernel"))) return st;
    lanczos_scale_kernel<<<grid, 256, 0, s>>>(n, w, nrm, 0, v);
    if ((st = check_launch("lanczos_scale_kernel"))) return st;
    for (int k = 0; k < iters; ++k) {
        lap_spmv_sell_kernel<<<grid, 256, 0, s>>>(n, S.sptr, S.perm, S.idx, S.val, g->strength, v, w, part);
        if ((st = check_launch("lap_spmv_sell_kernel"))) return st;
        lanczos_scalar_kernel<<<1, 256, 0, s>>>(part, grid, alpha, k, 0);
        if ((st = check_launch("lanczos_scalar_kernel"))) return st;
        if (k + 1 == iters) break;
        lanczos_update_kernel<<<grid, 256, 0, s>>>(n, w, v, vp, alpha, beta, k, part);
        if ((st = check_launch("lanczos_update_kernel"))) return st;
        lanczos_scalar_kernel<<<1, 256, 0, s>>>(part, grid, beta, k, 1);
        if ((st = check_launch("lanczos_scalar_kernel"))) return st;
        // vp <- v, v <- w / beta_k (rotate buffers: the old vp becomes the new v)
        std::swap(vp, v);
        lanczos_scale_kernel<<<grid, 256, 0, s>>>(n, w, beta, k, v);
        if ((st = check_launch("lanczos_scale_kernel"))) return st;
    }
    std::vector<double> a((size_t)iters), b((size_t)iters);
    SF_CHECK_CUDA(cudaMemcpyAsync(a.data(), alpha, sizeof(double) * iters, cudaMemcpyDeviceToHost, s));
    SF_CHECK_CUDA(cudaMemcpyAsync(b.data(), beta, sizeof(double) * iters, cudaMemcpyDeviceToHost, s));
    SF_CHECK_CUDA(cudaStreamSynchronize(s));
    // keep the leading part of the tridiagonal before the Krylov space is exhausted
    int k = iters;
    double scale = 0.0;
    for (int j = 0; j < iters; ++j) {
        if (!isfinite(a[j])) {
            k = j;
            break;
        }
        scale = fmax(scale, fabs(a[j]));
        if (j + 1 < iters) {
            if (!isfinite(b[j]) || b[j] <= 1e-12 * fmax(scale, b[j])) {
                k = j + 1;
                break;
            }
            scale = fmax(scale, b[j]);
        }
    }
    if (k < 1) {
        set_error("Lanczos produced no finite coefficient (graph values not finite?)");
        return SF_ERR_NUMERIC;
    }
    const double th = tridiag_max_eig_host(k, a.data(), b.data());
    if (theta_max) *theta_max = th;
    if (lam_hat) {
        double lh = fmin(1.01 * th, 2.0 * g->max_strength);
        *lam_hat = lh > 0.0 ? lh : 1.0;
    }
    return SF_OK;
}

SF_API sf_status sf_features(const float *Y, int32_t n, int32_t n_sig, int32_t normalize, float *F,
                             void *stream) {
    SF_ARG(Y && F, "Y/F is NULL");
    SF_ARG(n >= 0 && n_sig >= 1, "need n >= 0 and n_sig >= 1");
    if (n == 0) return SF_OK;
    cudaStream_t s = (cudaStream_t)stream;
    int64_t warps = n;
    int64_t grid = (warps * 32 + 255) / 256;
    const int64_t cap = (int64_t)sm_count() * 8;
    if (grid > cap) grid = cap;
    features_kernel<<<(unsigned)grid, 256, 0, s>>>(Y, n, n_sig, normalize, F);
    return check_launch("features_kernel");
}

}  // extern "C"
