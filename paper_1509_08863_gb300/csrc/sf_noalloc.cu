// Allocation-free variant of the moment sweep (sf_cheb_moments).
//
// Some callers cannot allocate device memory at the moment they need the
// eigenvalue-count moments: frameworks that hand the whole device memory to
// their own caching allocator and forbid foreign allocations, and
// latency-bound loops for which an allocator call (which may block, or, for
// cudaFree, synchronise the device) costs too much. This entry point serves
// them: all of its working memory is carved from one fixed array that lives
// in this library's device image, so the call itself never allocates.
//
// The array is a file-scope __device__ object of kNoAllocBytes; every GPU
// that loads the library keeps it until the process exits. Host code cannot
// use its name as a device address: the address is looked up once per device
// (cudaGetSymbolAddress, with that device current) by the first call made on
// that device, so that first call should come before any stream capture. All
// calls share the array and it keeps the previous call's contents, so
// everything that must start at zero is cleared on each call, and calls whose
// GPU work overlaps (different streams without ordering) race on it.
#include <math.h>

#include "sf_step.cuh"

namespace sf {

constexpr size_t kNoAllocBytes = 64ull << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

static std::mutex g_noalloc_mu;
static unsigned char *g_noalloc_ptr[64] = {nullptr};

// Device address of the array for the current device (looked up once per device).
static sf_status noalloc_base(unsigned char **out) {
    const int d = current_device();
    SF_ARG(d >= 0 && d < 64, "device index %d out of range", d);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[d]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_noalloc_ptr[d] = static_cast<unsigned char *>(p);
    }
    *out = g_noalloc_ptr[d];
    return SF_OK;
}

static size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

// Working memory of one call: 3 slab blocks of rows + 1 rows, d~ per slice
// row, partial sums, the per-order dot products and the sweep's block counter.
struct NoAllocPlan {
    size_t blk, dtil, part, dots, done, total;
};
static NoAllocPlan noalloc_plan(int64_t rows, int ld, int grid, int pack_grid, int p) {
    NoAllocPlan q;
    q.blk = round256((size_t)(rows + 1) * ld * sizeof(float));
    q.dtil = round256((size_t)rows * sizeof(float));
    q.part = round256((size_t)(2 * grid + 2 * pack_grid + 2) * sizeof(double));
    q.dots = round256((size_t)2 * (p + 1) * sizeof(double));
    q.done = 256;
    q.total = 3 * q.blk + q.dtil + q.part + q.dots + q.done;
    return q;
}

}  // namespace sf

using namespace sf;

extern "C" SF_API sf_status sf_cheb_moments_noalloc(const sf_graph *g, double lam_max, const float *R, int32_t n_sig,
                                                    int32_t p, double *moments, void *stream) {
    SF_ARG(g, "graph is NULL");
    SF_ARG(lam_max > 0.0 && isfinite(lam_max), "lam_max must be finite and > 0 (got %g)", lam_max);
    SF_ARG(p >= 0 && p <= 100000, "p must be in [0, 100000] (got %d)", p);
    SF_ARG(n_sig >= 1, "n_sig must be >= 1 (got %d)", n_sig);
    SF_ARG(R && moments, "R/moments is NULL");
    SF_ARG(g->device == current_device(), "graph lives on device %d, current device is %d", g->device,
           current_device());
    {
        std::lock_guard<std::mutex> lk(g->sell_mu);
        SF_ARG(g->sell.built,
               "the graph has no sweep layout yet: call sf_cheb_moments or sf_cheb_filter on it once, where "
               "allocation is allowed");
    }
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char *base = nullptr;
    sf_status st = noalloc_base(&base);
    if (st) return st;

    const int64_t n = g->n;
    const int64_t rows = g->sell.rows;
    const int32_t *perm = g->sell.perm;
    const bool weighted = !g->unit_weights;
    const int pack_grid = kPackBlocksPerSm * sm_count();
    // The slab sf_cheb_moments picks by default, halved (down to 8 columns) until
    // the working memory fits the array: the size limit is monotone in N.
    int ld = auto_slab_cols(n, n_sig, SF_F32, 32ll << 20);
    SweepShape sh;
    NoAllocPlan plan;
    for (;;) {
        if ((st = make_shape(SF_F32, ld, 0, 0, MODE_MOM, weighted, &sh, 0))) return st;
        plan = noalloc_plan(rows, ld, sh.grid, pack_grid, p);
        if (plan.total <= kNoAllocBytes || ld <= 8) break;
        ld /= 2;
    }
    SF_ARG(plan.total <= kNoAllocBytes,
           "this graph and signal count need %zu bytes of working memory; the allocation-free variant has %zu",
           plan.total, kNoAllocBytes);
    SF_ARG((int64_t)(rows + 1) * ld < (1ll << 32), "graph too large for 32-bit slab offsets");

    float *buf[3];
    size_t off = 0;
    for (int k = 0; k < 3; ++k) {
        buf[k] = reinterpret_cast<float *>(base + off);
        off += plan.blk;
    }
    float *dtil = reinterpret_cast<float *>(base + off);
    off += plan.dtil;
    double *part = reinterpret_cast<double *>(base + off);
    off += plan.part;
    double *dots = reinterpret_cast<double *>(base + off);
    off += plan.dots;
    uint32_t *done = reinterpret_cast<uint32_t *>(base + off);

    // the array keeps the last call's contents: clear the accumulators, the block
    // counter and the zero rows
    SF_CHECK_CUDA(cudaMemsetAsync(dots, 0, plan.dots, s));
    SF_CHECK_CUDA(cudaMemsetAsync(done, 0, sizeof(uint32_t), s));
    for (int k = 0; k < 3; ++k)
        SF_CHECK_CUDA(cudaMemsetAsync(buf[k] + (size_t)rows * ld, 0, (size_t)ld * sizeof(float), s));
    if (rows > 0) {
        dtil_kernel<<<(unsigned)((rows + 255) / 256), 256, 0, s>>>(g->strength, (int32_t)rows, 2.0 / lam_max,
                                                                   nullptr, nullptr, dtil, nullptr, perm, nullptr);
        if ((st = check_launch("dtil_kernel"))) return st;
    }
    int32_t *status = device_status();
    SF_ARG(status, "device status word unavailable");
    for (int c0 = 0; c0 < n_sig; c0 += ld) {
        const int w = (n_sig - c0) < ld ? (n_sig - c0) : ld;
        pack_kernel<float><<<pack_grid, 256, 0, s>>>(R, SF_F32, (int32_t)n, n_sig, c0, w, ld, buf[0], nullptr, 0, 0,
                                                     nullptr, 1, 0, nullptr, nullptr, part, nullptr, perm,
                                                     (int32_t)rows);
        if ((st = check_launch("pack_kernel"))) return st;
        pair_sum_kernel<<<1, 256, 0, s>>>(part, pack_grid, 1, dots);
        if ((st = check_launch("pair_sum_kernel"))) return st;
        StepParams P = {};
        P.n = (int32_t)n;
        P.sell_ptr = g->sell.sptr;
        P.sell_idx = g->sell.ridx;
        P.sell_val = g->sell.val;
        P.dtil = dtil;
        P.wscale_u = (float)(2.0 / lam_max);
        P.ld = ld;
        P.flags = kStepFlagsDefault;
        P.part = part;
        P.done = done;
        P.status = status;
        for (int j = 1; j <= p; ++j) {
            P.X = buf[(j - 1) % 3];
            P.Z = (j >= 2) ? buf[(j - 2) % 3] : nullptr;
            P.out = buf[j % 3];
            P.m = (j == 1) ? 1.0f : 2.0f;
            P.j = j;
            P.dots = dots + 2 * j;  // the kernel's last block adds <T_j,T_j>, <T_j,T_{j-1}>
            if ((st = launch_step(sh, MODE_MOM, P, s, 0.0))) return st;
        }
    }
    // dots = [D_0, E_0, D_1, E_1, ..., D_p, E_p] with D_j = <T_j, T_j>, E_j = <T_j, T_{j-1}>;
    // copy the first 2p + 1 straight into the caller's array, check them as
    // sf_cheb_moments does, and convert in place:
    // mu_0 = D_0, mu_1 = E_1, mu_2j = 2 D_j - mu_0, mu_{2j-1} = 2 E_j - mu_1 (j >= 2)
    double last = 0.0;
    SF_CHECK_CUDA(cudaMemcpyAsync(moments, dots, sizeof(double) * (size_t)(2 * p + 1), cudaMemcpyDeviceToHost, s));
    SF_CHECK_CUDA(cudaMemcpyAsync(&last, dots + 2 * p + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
    SF_CHECK_CUDA(cudaStreamSynchronize(s));
    if ((st = sf_device_check(stream))) return st;
    if ((st = check_moment_dots(moments, last, p, lam_max))) return st;
    if (p >= 1) {
        const double mu0 = moments[0];
        const double mu1 = (p == 1) ? last : moments[3];
        for (int j = 1; j <= p; ++j) moments[2 * j] = 2.0 * moments[2 * j] - mu0;
        for (int j = 2; j <= p; ++j) {
            const double e = (2 * j + 1 == 2 * p + 1) ? last : moments[2 * j + 1];
            moments[2 * j - 1] = 2.0 * e - mu1;
        }
        moments[1] = mu1;
    }
    return SF_OK;
}
