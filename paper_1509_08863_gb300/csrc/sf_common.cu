// Status handling, allocation, scans and reductions, host-side FP64 math
// (coefficients, counts from moments, dichotomy), profiling hooks.
#include <math.h>

#include <vector>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <mutex>

#include "sf_internal.cuh"

namespace sf {

static thread_local char g_err[512] = "";
static std::atomic<int64_t> g_launches{0};

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

sf_status cuda_fail(cudaError_t e, const char *what) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? SF_ERR_OOM : SF_ERR_CUDA;
}

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

sf_status check_launch(const char *name) {
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, name);
    return SF_OK;
}

sf_status dev_alloc(void **p, size_t bytes, cudaStream_t s) {
    *p = nullptr;
    if (bytes == 0) return SF_OK;
    cudaError_t e = cudaMallocAsync(p, bytes, s);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        set_error("device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
        return SF_ERR_OOM;
    }
    return SF_OK;
}

void dev_free(void *p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

int current_device() {
    int d = 0;
    cudaGetDevice(&d);
    return d;
}

int sm_count() {
    static int cache[64] = {0};
    int d = current_device();
    if (d < 64 && cache[d]) return cache[d];
    int c = 0;
    cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, d);
    if (c <= 0) c = 1;
    if (d < 64) cache[d] = c;
    return c;
}

// ---------------------------------------------------------------- scan
// Block scan of 2048 int32 (256 threads x 8 items), exclusive.
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__global__ void scan_tile_kernel(const int32_t *in, int32_t *out, int32_t *tile_sums, int64_t n) {
    __shared__ int32_t warp_tot[kScanThreads / 32];
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int32_t v[kScanItems];
    int32_t run = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t idx = base + k;
        int32_t x = idx < n ? in[idx] : 0;
        v[k] = run;
        run += x;
    }
    // inclusive warp scan of per-thread totals
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int32_t inc = run;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        int32_t y = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += y;
    }
    if (lane == 31) warp_tot[w] = inc;
    __syncthreads();
    if (w == 0) {
        int32_t t = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
        int32_t ti = t;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            int32_t y = __shfl_up_sync(0xffffffffu, ti, off);
            if (lane >= off) ti += y;
        }
        if (lane < kScanThreads / 32) warp_tot[lane] = ti - t;  // exclusive
        if (lane == kScanThreads / 32 - 1 && tile_sums) tile_sums[blockIdx.x] = ti;
    }
    __syncthreads();
    int32_t off = warp_tot[w] + inc - run;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t idx = base + k;
        if (idx < n) out[idx] = v[k] + off;
    }
}

__global__ void scan_add_kernel(int32_t *out, const int32_t *tile_offs, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += tile_offs[i / kScanTile];
}

sf_status exclusive_scan_i32(const int32_t *in, int32_t *out, int64_t n, cudaStream_t s) {
    if (n <= 0) return SF_OK;
    int64_t tiles = (n + kScanTile - 1) / kScanTile;
    if (tiles == 1) {
        scan_tile_kernel<<<1, kScanThreads, 0, s>>>(in, out, nullptr, n);
        return check_launch("scan_tile_kernel");
    }
    Scratch sc(s);
    int32_t *sums = nullptr;
    sf_status st = sc.get(&sums, (size_t)tiles);
    if (st) return st;
    scan_tile_kernel<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, out, sums, n);
    if ((st = check_launch("scan_tile_kernel"))) return st;
    if ((st = exclusive_scan_i32(sums, sums, tiles, s))) return st;
    scan_add_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(out, sums, n);
    return check_launch("scan_add_kernel");
}

// ---------------------------------------------------------------- f64 sum
// One block sums a strided slice; a second pass sums the block results, both
// in a fixed order, so the result does not depend on scheduling.
__global__ void sum_f64_kernel(const double *in, int64_t count, double *out) {
    __shared__ double sh[256];
    double acc = 0.0;
    int64_t per = (count + gridDim.x - 1) / gridDim.x;
    int64_t beg = (int64_t)blockIdx.x * per, end = beg + per < count ? beg + per : count;
    for (int64_t i = beg + threadIdx.x; i < end; i += blockDim.x) acc += in[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = sh[0];
}

sf_status reduce_sum_f64(const double *in, int64_t count, double *out, cudaStream_t s) {
    if (count <= 65536) {
        sum_f64_kernel<<<1, 256, 0, s>>>(in, count, out);
        return check_launch("sum_f64_kernel");
    }
    Scratch sc(s);
    double *part = nullptr;
    sf_status st = sc.get(&part, 256);
    if (st) return st;
    sum_f64_kernel<<<256, 256, 0, s>>>(in, count, part);
    if ((st = check_launch("sum_f64_kernel"))) return st;
    sum_f64_kernel<<<1, 256, 0, s>>>(part, 256, out);
    return check_launch("sum_f64_kernel");
}

// ---------------------------------------------------------------- host math
// Chebyshev projection of the ideal low-pass of Eq. (2): with
// x = 2 lambda / lam_max - 1 and theta_c = arccos(x_c), the integral
// (2/pi) int_{theta_c}^{pi} cos(j t) dt gives c_0 = 2 (1 - theta_c/pi) and
// c_j = -2 sin(j theta_c) / (pi j); the series takes c_0 / 2. Jackson
// factors g_j = [(p+2-j) cos(pi j/(p+2)) + sin(pi j/(p+2)) cot(pi/(p+2))]/(p+2).
void cheb_coeffs_host(double lam_max, double lc, int p, int jackson, double *a) {
    const double pi = 3.14159265358979323846;
    double xc = 2.0 * lc / lam_max - 1.0;
    xc = xc > 1.0 ? 1.0 : (xc < -1.0 ? -1.0 : xc);
    double tc = acos(xc);
    double q = (double)(p + 2);
    double cot1 = cos(pi / q) / sin(pi / q);
    for (int j = 0; j <= p; ++j) {
        double c = (j == 0) ? 1.0 - tc / pi : -2.0 * sin(j * tc) / (pi * j);
        if (jackson) c *= ((q - j) * cos(pi * j / q) + sin(pi * j / q) * cot1) / q;
        a[j] = c;
    }
}

// ||F R||_F^2 = sum_{j,j'} a_j a_j' <T_j R, T_j' R> and T_j T_j' = (T_{j+j'} + T_{|j-j'|})/2.
// Rewritten with symmetric weights: sum_j a_j^2 (mu_2j + mu_0)/2 + sum_{j<j'} a_j a_j' (mu_{j+j'} + mu_{j'-j}).
double count_from_moments_host(const double *mu, int p, const double *a) {
    double s = 0.0;
    for (int j = 0; j <= p; ++j) {
        s += a[j] * a[j] * 0.5 * (mu[2 * j] + mu[0]);
        for (int jj = j + 1; jj <= p; ++jj) s += a[j] * a[jj] * (mu[j + jj] + mu[jj - j]);
    }
    return s;
}

// Largest eigenvalue of a symmetric tridiagonal by Sturm-count bisection.
static int sturm_below(int k, const double *a, const double *b, double x) {
    int c = 0;
    double d = 1.0;
    for (int i = 0; i < k; ++i) {
        double t = (i == 0) ? 0.0 : b[i - 1] * b[i - 1] / d;
        d = (a[i] - x) - t;
        if (d == 0.0) d = -1e-300;
        if (d < 0.0) ++c;
    }
    return c;
}

double tridiag_max_eig_host(int k, const double *a, const double *b) {
    double lo = a[0], hi = a[0];
    for (int i = 0; i < k; ++i) {
        double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i + 1 < k ? fabs(b[i]) : 0.0);
        lo = fmin(lo, a[i] - r);
        hi = fmax(hi, a[i] + r);
    }
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (sturm_below(k, a, b, mid) >= k) hi = mid;
        else lo = mid;
    }
    return hi;
}

// ---------------------------------------------------------------- profiling
struct ProfRec {
    int ev;            // index of the first event of the pair
    double bytes;      // algorithmic bytes of the launches
    int tag;           // kernel variant
    int64_t launches;  // launches between the two events
};
struct ProfTotals {
    int64_t launches = 0;
    double ms = 0.0, bytes = 0.0;
};
struct ProfState {
    std::mutex mu;
    bool on = false;
    std::vector<cudaEvent_t> pool;
    std::vector<ProfRec> recs;
    size_t used = 0;
    ProfTotals last[kProfTags];  // per-variant totals of the last sf_profile_end
};
static ProfState &prof() {
    static ProfState p;
    return p;
}

bool profiling_on() { return prof().on; }

bool profile_events(cudaEvent_t *a, cudaEvent_t *b) {
    ProfState &P = prof();
    std::lock_guard<std::mutex> lk(P.mu);
    if (!P.on) return false;
    while (P.pool.size() < P.used + 2) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return false;
        P.pool.push_back(e);
    }
    *a = P.pool[P.used];
    *b = P.pool[P.used + 1];
    return true;
}

void profile_record(cudaEvent_t a, cudaEvent_t b, double bytes, int tag, int64_t launches) {
    ProfState &P = prof();
    std::lock_guard<std::mutex> lk(P.mu);
    (void)a;
    (void)b;
    P.recs.push_back({(int)P.used, bytes, (tag >= 0 && tag < kProfTags) ? tag : 0, launches});
    P.used += 2;
}

static thread_local bool t_span = false;
bool profile_span_active() { return t_span; }
void profile_span_set(bool on) { t_span = on; }

}  // namespace sf

using namespace sf;

extern "C" {

SF_API const char *sf_status_str(sf_status s) {
    switch (s) {
        case SF_OK: return "SF_OK";
        case SF_ERR_ARG: return "SF_ERR_ARG: invalid argument";
        case SF_ERR_CUDA: return "SF_ERR_CUDA: CUDA failure";
        case SF_ERR_OOM: return "SF_ERR_OOM: device allocation failed";
        case SF_ERR_TIMEOUT: return "SF_ERR_TIMEOUT: bounded device wait gave up";
        case SF_ERR_NUMERIC: return "SF_ERR_NUMERIC: non-finite value";
        default: return "unknown status";
    }
}

SF_API const char *sf_last_error(void) { return g_err; }

SF_API int32_t sf_version(void) { return 100; }

SF_API int64_t sf_launch_count(void) { return g_launches.load(); }

SF_API sf_status sf_cheb_coeffs(double lam_max, const double *cutoffs, int32_t n_cut, int32_t p,
                                int32_t jackson, double *coeffs) {
    SF_ARG(lam_max > 0.0 && isfinite(lam_max), "lam_max must be finite and > 0 (got %g)", lam_max);
    SF_ARG(n_cut >= 1 && p >= 0, "need n_cut >= 1 and p >= 0");
    SF_ARG(cutoffs && coeffs, "null pointer");
    for (int c = 0; c < n_cut; ++c) {
        SF_ARG(isfinite(cutoffs[c]), "cutoff %d is not finite", c);
        cheb_coeffs_host(lam_max, cutoffs[c], p, jackson, coeffs + (int64_t)c * (p + 1));
    }
    return SF_OK;
}

SF_API sf_status sf_count_from_moments(const double *moments, int32_t p, const double *coeffs,
                                       int32_t n_cut, double *counts) {
    SF_ARG(moments && coeffs && counts, "null pointer");
    SF_ARG(p >= 0 && n_cut >= 1, "need p >= 0 and n_cut >= 1");
    for (int c = 0; c < n_cut; ++c)
        counts[c] = count_from_moments_host(moments, p, coeffs + (int64_t)c * (p + 1));
    return SF_OK;
}

SF_API sf_status sf_dichotomy(const double *moments, int32_t p, double lam_max, double k, int32_t jackson,
                              int32_t max_iter, double tol, double *lam_k) {
    SF_ARG(moments && lam_k, "null pointer");
    SF_ARG(p >= 0 && lam_max > 0.0, "need p >= 0 and lam_max > 0");
    std::vector<double> a((size_t)p + 1);
    double lo = 0.0, hi = lam_max;
    for (int it = 0; it < max_iter && (hi - lo) > tol * lam_max; ++it) {
        double mid = 0.5 * (lo + hi);
        cheb_coeffs_host(lam_max, mid, p, jackson, a.data());
        double cnt = count_from_moments_host(moments, p, a.data());
        if (cnt >= k) hi = mid;
        else lo = mid;
    }
    *lam_k = hi;
    return SF_OK;
}

SF_API sf_status sf_cheb_order(double x, double delta, double w, int32_t jackson, int32_t p_max, int32_t *m_star) {
    SF_ARG(m_star, "m_star is NULL");
    SF_ARG(x >= 0.0 && x <= 1.0, "x = lambda_c / lambda_N must lie in [0, 1]");
    SF_ARG(delta > 0.0 && w >= 0.0 && p_max >= 1 && p_max <= 100000, "need delta > 0, w >= 0, 1 <= p_max <= 100000");
    // evaluation points: the uniform grid g / 4095 and the band edges, outside the band |t - x| < w
    std::vector<double> pts;
    pts.reserve(4098);
    for (int gi = 0; gi < 4096; ++gi) pts.push_back((double)gi / 4095.0);
    if (x - w >= 0.0) pts.push_back(x - w);
    if (x + w <= 1.0) pts.push_back(x + w);
    std::vector<double> a((size_t)p_max + 1);
    *m_star = -1;
    for (int m = 1; m <= p_max; ++m) {
        cheb_coeffs_host(1.0, x, m, jackson, a.data());
        double worst = 0.0;
        for (double t : pts) {
            if (fabs(t - x) < w) continue;
            // Clenshaw: b_j = a_j + 2 y b_{j+1} - b_{j+2}; P = a_0 + y b_1 - b_2
            const double y = 2.0 * t - 1.0;
            double b1 = 0.0, b2 = 0.0;
            for (int j = m; j >= 1; --j) {
                const double b0 = a[j] + 2.0 * y * b1 - b2;
                b2 = b1;
                b1 = b0;
            }
            const double v = a[0] + y * b1 - b2;
            const double e = fabs((t <= x ? 1.0 : 0.0) - v);
            if (e > worst) worst = e;
        }
        if (worst <= delta) {
            *m_star = m;
            break;
        }
    }
    return SF_OK;
}

SF_API sf_status sf_profile_begin(void) {
    ProfState &P = prof();
    std::lock_guard<std::mutex> lk(P.mu);
    P.on = true;
    P.used = 0;
    P.recs.clear();
    return SF_OK;
}

SF_API sf_status sf_profile_variant(int32_t tag, int64_t *launches, double *ms, double *bytes) {
    SF_ARG(tag >= 0 && tag < kProfTags, "tag must be in [0, %d)", kProfTags);
    ProfState &P = prof();
    std::lock_guard<std::mutex> lk(P.mu);
    if (launches) *launches = P.last[tag].launches;
    if (ms) *ms = P.last[tag].ms;
    if (bytes) *bytes = P.last[tag].bytes;
    return SF_OK;
}

SF_API sf_status sf_profile_end(int64_t *launches, double *ms, double *bytes) {
    ProfState &P = prof();
    std::lock_guard<std::mutex> lk(P.mu);
    P.on = false;
    double tot = 0.0, by = 0.0;
    int64_t n_launch = 0;
    for (auto &t : P.last) t = ProfTotals();
    for (auto &r : P.recs) {
        cudaEvent_t a = P.pool[r.ev], b = P.pool[r.ev + 1];
        cudaError_t e = cudaEventSynchronize(b);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
        float t = 0.f;
        e = cudaEventElapsedTime(&t, a, b);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime");
        tot += t;
        by += r.bytes;
        n_launch += r.launches;
        P.last[r.tag].launches += r.launches;
        P.last[r.tag].ms += t;
        P.last[r.tag].bytes += r.bytes;
    }
    if (launches) *launches = n_launch;
    if (ms) *ms = tot;
    if (bytes) *bytes = by;
    P.recs.clear();
    P.used = 0;
    return SF_OK;
}

}  // extern "C"
