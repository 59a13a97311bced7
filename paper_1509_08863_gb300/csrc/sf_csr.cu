// Graph construction: symmetric CSR of W from an undirected edge list
// (§2: W_ij = W_ji >= 0), strengths s_i (§2.1), block-diagonal batches.
//
// Pipeline (all deterministic, so the CSR is bit-identical for any edge
// order and any scheduling):
//   1. expand: each edge (u, v) with u != v gives keys (u << cb | v) and
//      (v << cb | u); self-loops become a sentinel that sorts last.
//   2. LSD radix sort of the 64-bit keys (8-bit digits, stable scatter
//      computed from warp match masks) carrying the weights.
//   3. run heads of equal keys -> prefix sum -> one CSR entry per distinct
//      pair holding the largest weight of its run.
//   4. per-row counts -> prefix sum -> rowptr; strengths per row in FP64.
#include <math.h>

#include "sf_internal.cuh"

namespace sf {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 8;  // per thread
constexpr int kSortTile = kSortThreads * kSortItems;

__global__ void fill_i32_kernel(int32_t *p, int count, int32_t v) {
    if ((int)threadIdx.x < count) p[threadIdx.x] = v;
}

__global__ void expand_edges_kernel(const int32_t *src, const int32_t *dst, const float *w, int64_t m,
                                    int32_t n, int cb, uint64_t sentinel, uint64_t *keys, float *vals,
                                    int32_t *flags /* [0]=bad index [1]=bad weight [2]=self loops */) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m) return;
    int32_t u = src[e], v = dst[e];
    float x = w ? w[e] : 1.0f;
    bool bad = (u < 0 || u >= n || v < 0 || v >= n);
    if (bad) atomicOr(&flags[0], 1);
    if (!(x >= 0.0f) || isinf(x)) atomicOr(&flags[1], 1);
    if (bad || u == v) {
        if (!bad) atomicAdd(&flags[2], 1);
        keys[2 * e] = sentinel;
        keys[2 * e + 1] = sentinel;
        vals[2 * e] = 0.f;
        vals[2 * e + 1] = 0.f;
        return;
    }
    keys[2 * e] = ((uint64_t)u << cb) | (uint64_t)v;
    keys[2 * e + 1] = ((uint64_t)v << cb) | (uint64_t)u;
    vals[2 * e] = x;
    vals[2 * e + 1] = x;
}

// Per-tile digit histogram, written digit-major: hist[d * tiles + tile].
__global__ void radix_hist_kernel(const uint64_t *keys, int64_t count, int shift, int32_t *hist,
                                  int32_t tiles) {
    __shared__ int32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int k = threadIdx.x; k < kSortTile; k += kSortThreads) {
        int64_t idx = base + k;
        if (idx < count) atomicAdd(&h[(keys[idx] >> shift) & 0xFF], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * tiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter. Warp w owns items [w*256, (w+1)*256) of the tile and walks
// them in 8 rounds of 32 consecutive items; equal digits in a round are
// ranked by lane order through __match_any_sync, and running per-warp digit
// counts carry the order across rounds. Per-digit warp bases then follow
// warp order, so the scatter preserves input order among equal digits. The
// tile's items are first placed in shared memory in (digit, input) order,
// then written out by consecutive threads: each digit's items of a tile land
// in consecutive words (coalesced runs) instead of one scattered word per
// item.
__global__ void radix_scatter_kernel(const uint64_t *keys_in, const float *vals_in, uint64_t *keys_out,
                                     float *vals_out, int64_t count, int shift, const int32_t *offs,
                                     int32_t tiles) {
    __shared__ int32_t wcnt[kSortWarps][256];
    __shared__ int32_t tdig[256];  // first tile-local position of each digit
    __shared__ int32_t wsum[kSortWarps];
    __shared__ uint64_t s_key[kSortTile];
    __shared__ float s_val[kSortTile];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int d = lane; d < 256; d += 32) wcnt[w][d] = 0;
    __syncwarp();
    const int64_t tile0 = (int64_t)blockIdx.x * kSortTile;
    const int64_t base = tile0 + (int64_t)w * 256;
    uint64_t key[kSortItems];
    float val[kSortItems];
    int32_t rank[kSortItems];
    int32_t dig[kSortItems];
    const unsigned lt_mask = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        int64_t idx = base + r * 32 + lane;
        bool ok = idx < count;
        key[r] = ok ? keys_in[idx] : 0ull;
        val[r] = (ok && vals_in) ? vals_in[idx] : 0.f;
        int d = ok ? (int)((key[r] >> shift) & 0xFF) : 256 + lane;  // out-of-range items never match
        dig[r] = ok ? d : -1;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int before = ok ? wcnt[w][d] : 0;
        __syncwarp();
        if (ok && (peers & lt_mask) == 0) wcnt[w][d] = before + __popc(peers);
        __syncwarp();
        rank[r] = before + __popc(peers & lt_mask);
    }
    __syncthreads();
    // exclusive prefix over warps, one digit per thread, then over digits
    {
        const int d = threadIdx.x;
        int32_t run = 0;
#pragma unroll
        for (int q = 0; q < kSortWarps; ++q) {
            int32_t c = wcnt[q][d];
            wcnt[q][d] = run;
            run += c;
        }
        int32_t v = run;  // inclusive scan of the digit totals within the warp
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, v, off);
            if (lane >= off) v += y;
        }
        if (lane == 31) wsum[w] = v;
        __syncthreads();
        int32_t wb = 0;
        for (int q = 0; q < w; ++q) wb += wsum[q];
        tdig[d] = wb + v - run;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        if (dig[r] < 0) continue;
        const int d = dig[r];
        const int32_t lp = tdig[d] + wcnt[w][d] + rank[r];
        s_key[lp] = key[r];
        if (vals_out) s_val[lp] = val[r];
    }
    __syncthreads();
    const int items = (int)min((int64_t)kSortTile, count - tile0);
    for (int t = threadIdx.x; t < items; t += kSortThreads) {
        const uint64_t kk = s_key[t];
        const int d = (int)((kk >> shift) & 0xFF);
        const int64_t pos = (int64_t)offs[(int64_t)d * tiles + blockIdx.x] + (t - tdig[d]);
        keys_out[pos] = kk;
        if (vals_out) vals_out[pos] = s_val[t];
    }
}

// head[i] = 1 where a run of equal keys starts (i < valid).
__global__ void run_heads_kernel(const uint64_t *keys, int64_t valid, int32_t *head) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= valid) return;
    head[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
}

// For each run head: colidx/val at the run's output slot (largest weight of
// the run) and one count for its row.
// The keys are sorted, so a warp's heads mostly share one or two rows: the
// row counts are added once per row and warp (the lanes of a row matched).
__global__ void compact_runs_kernel(const uint64_t *keys, const float *vals, const int32_t *head,
                                    const int32_t *pos, int64_t valid, int cb, int32_t *colidx, float *val,
                                    int32_t *rowcnt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const bool h = i < valid && head[i];
    int32_t row = -1 - lane;  // distinct for lanes without a head: they match no other lane
    if (h) {
        const uint64_t k = keys[i];
        float x = vals[i];
        for (int64_t t = i + 1; t < valid && keys[t] == k; ++t) x = fmaxf(x, vals[t]);
        const int32_t o = pos[i];
        colidx[o] = (int32_t)(k & ((1ull << cb) - 1ull));
        val[o] = x;
        row = (int32_t)(k >> cb);
    }
    const unsigned peers = __match_any_sync(0xffffffffu, row);
    if (h && lane == __ffs(peers) - 1) atomicAdd(&rowcnt[row], __popc(peers));
}

// s_i = sum of row i in column order (FP64); flags[0] set if a weight != 1;
// the largest s_i. The flag and the maximum are combined over the warp first
// (one atomic per warp instead of one per row on a single address).
__global__ void strength_kernel(int32_t n, const int32_t *rowptr, const float *val, double *s,
                                int32_t *nonunit, unsigned long long *smax_bits) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    double acc = 0.0;
    int nu = 0;
    if (i < n) {
        for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
            float x = val[e];
            acc += (double)x;
            nu |= (x != 1.0f);
        }
        s[i] = acc;
    }
    // non-negative doubles order like their bit patterns
    unsigned long long m = (unsigned long long)__double_as_longlong(acc);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, m, off);
        m = o > m ? o : m;
    }
    const bool any_nu = __any_sync(0xffffffffu, nu);
    if ((threadIdx.x & 31) == 0) {
        if (any_nu) atomicOr(nonunit, 1);
        atomicMax(smax_bits, m);
    }
}

sf_status compute_strength(sf_graph *g, cudaStream_t s) {
    Scratch sc(s);
    int32_t *flag = nullptr;
    unsigned long long *smax = nullptr;
    sf_status st;
    if ((st = sc.get(&flag, 1))) return st;
    if ((st = sc.get(&smax, 1))) return st;
    SF_CHECK_CUDA(cudaMemsetAsync(flag, 0, sizeof(int32_t), s));
    SF_CHECK_CUDA(cudaMemsetAsync(smax, 0, sizeof(unsigned long long), s));
    strength_kernel<<<(g->n + 255) / 256, 256, 0, s>>>(g->n, g->rowptr, g->val, g->strength, flag, smax);
    if ((st = check_launch("strength_kernel"))) return st;
    int32_t hflag = 0;
    unsigned long long hmax = 0;
    SF_CHECK_CUDA(cudaMemcpyAsync(&hflag, flag, sizeof(hflag), cudaMemcpyDeviceToHost, s));
    SF_CHECK_CUDA(cudaMemcpyAsync(&hmax, smax, sizeof(hmax), cudaMemcpyDeviceToHost, s));
    SF_CHECK_CUDA(cudaStreamSynchronize(s));
    g->unit_weights = hflag ? 0 : 1;
    double m;
    memcpy(&m, &hmax, sizeof(m));
    g->max_strength = m;
    return SF_OK;
}

sf_status radix_sort(uint64_t *&keys, float *&vals, uint64_t *&keys_alt, float *&vals_alt, int64_t count,
                     int shift0, int bits, cudaStream_t s) {
    if (count <= 1) return SF_OK;
    int32_t tiles = (int32_t)((count + kSortTile - 1) / kSortTile);
    Scratch sc(s);
    int32_t *hist = nullptr;
    sf_status st = sc.get(&hist, (size_t)tiles * 256);
    if (st) return st;
    for (int shift = shift0; shift < bits; shift += 8) {
        radix_hist_kernel<<<tiles, kSortThreads, 0, s>>>(keys, count, shift, hist, tiles);
        if ((st = check_launch("radix_hist_kernel"))) return st;
        if ((st = exclusive_scan_i32(hist, hist, (int64_t)tiles * 256, s))) return st;
        radix_scatter_kernel<<<tiles, kSortThreads, 0, s>>>(keys, vals, keys_alt, vals_alt, count, shift, hist,
                                                            tiles);
        if ((st = check_launch("radix_scatter_kernel"))) return st;
        std::swap(keys, keys_alt);
        std::swap(vals, vals_alt);
    }
    return SF_OK;
}

// Normalised Laplacian I - S^-1/2 W S^-1/2 (the footnote of §2.1): weights
// w_ij / sqrt(s_i s_j) computed in FP64 and rounded to FP32, diagonal 1 (0 for
// an isolated node). One thread per row.
__global__ void normalize_kernel(int32_t n, const int32_t *rowptr, const int32_t *colidx, const float *val,
                                 const double *s, float *val_out, double *diag_out, int32_t *any) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double si = s[i];
    diag_out[i] = si > 0.0 ? 1.0 : 0.0;
    if (si > 0.0) *any = 1;
    for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
        const double ss = si * s[colidx[e]];
        const double w = val ? (double)val[e] : 1.0;
        val_out[e] = ss > 0.0 ? (float)(w / sqrt(ss)) : 0.0f;
    }
}

static void graph_release(sf_graph *g) {
    if (!g) return;
    sell_release(&g->sell);
    cudaFree(g->rowptr);
    cudaFree(g->colidx);
    cudaFree(g->val);
    cudaFree(g->strength);
    delete g;
}

}  // namespace sf

using namespace sf;

extern "C" {

SF_API sf_status sf_csr_build(int32_t n_nodes, int64_t n_edges, const int32_t *src, const int32_t *dst,
                              const float *w, void *stream, sf_graph **out) {
    SF_ARG(out, "out is NULL");
    *out = nullptr;
    SF_ARG(n_nodes >= 1, "n_nodes must be >= 1 (got %d)", n_nodes);
    SF_ARG(n_edges >= 0, "n_edges must be >= 0");
    SF_ARG(2 * n_edges < (int64_t)INT32_MAX, "2 * n_edges must be < 2^31 (got %lld edges)", (long long)n_edges);
    SF_ARG(n_edges == 0 || (src && dst), "src/dst are NULL");
    cudaStream_t s = (cudaStream_t)stream;
    int cb = 1;
    while ((1ll << cb) < (int64_t)n_nodes) ++cb;
    const int bits = 2 * cb;
    const uint64_t sentinel = (bits >= 64) ? ~0ull : ((1ull << bits) - 1ull);
    const int64_t cnt = 2 * n_edges;

    sf_graph *g = new sf_graph();
    g->n = n_nodes;
    g->device = current_device();
    sf_status st = SF_OK;
    auto fail = [&](sf_status e) {
        graph_release(g);
        return e;
    };
    if (cudaMalloc(&g->rowptr, sizeof(int32_t) * (size_t)(n_nodes + 1 + kCsrPad)) != cudaSuccess ||
        cudaMalloc(&g->strength, sizeof(double) * (size_t)n_nodes) != cudaSuccess) {
        cudaGetLastError();
        set_error("device allocation failed for a graph of %d nodes", n_nodes);
        return fail(SF_ERR_OOM);
    }
    {
        Scratch sc(s);
        uint64_t *k0 = nullptr, *k1 = nullptr;
        float *v0 = nullptr, *v1 = nullptr;
        int32_t *flags = nullptr, *head = nullptr, *rowcnt = nullptr;
        if ((st = sc.get(&flags, 3))) return fail(st);
        if ((st = sc.get(&rowcnt, (size_t)n_nodes + 1))) return fail(st);
        if (cnt > 0) {
            if ((st = sc.get(&k0, (size_t)cnt)) || (st = sc.get(&k1, (size_t)cnt)) ||
                (st = sc.get(&v0, (size_t)cnt)) || (st = sc.get(&v1, (size_t)cnt)) ||
                (st = sc.get(&head, (size_t)cnt)))
                return fail(st);
        }
        if (cudaMemsetAsync(flags, 0, 3 * sizeof(int32_t), s) != cudaSuccess ||
            cudaMemsetAsync(rowcnt, 0, sizeof(int32_t) * (size_t)(n_nodes + 1), s) != cudaSuccess)
            return fail(cuda_fail(cudaGetLastError(), "cudaMemsetAsync"));
        int64_t valid = 0, nnz = 0;
        if (n_edges > 0) {
            expand_edges_kernel<<<(unsigned)((n_edges + 255) / 256), 256, 0, s>>>(src, dst, w, n_edges, n_nodes,
                                                                                  cb, sentinel, k0, v0, flags);
            if ((st = check_launch("expand_edges_kernel"))) return fail(st);
            int32_t hf[3];
            if (cudaMemcpyAsync(hf, flags, sizeof(hf), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                return fail(cuda_fail(cudaGetLastError(), "reading edge checks"));
            if (hf[0]) {
                set_error("edge endpoint outside [0, %d)", n_nodes);
                return fail(SF_ERR_ARG);
            }
            if (hf[1]) {
                set_error("negative or non-finite edge weight");
                return fail(SF_ERR_ARG);
            }
            valid = cnt - 2 * (int64_t)hf[2];
            if ((st = radix_sort(k0, v0, k1, v1, cnt, 0, bits, s))) return fail(st);
            if (valid > 0) {
                run_heads_kernel<<<(unsigned)((valid + 255) / 256), 256, 0, s>>>(k0, valid, head);
                if ((st = check_launch("run_heads_kernel"))) return fail(st);
                int32_t last_head = 0, last_pos = 0;
                if (cudaMemcpyAsync(&last_head, head + valid - 1, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess)
                    return fail(cuda_fail(cudaGetLastError(), "cudaMemcpyAsync"));
                int32_t *pos = (int32_t *)k1;  // reuse the alternate key buffer
                if ((st = exclusive_scan_i32(head, pos, valid, s))) return fail(st);
                if (cudaMemcpyAsync(&last_pos, pos + valid - 1, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                    cudaStreamSynchronize(s) != cudaSuccess)
                    return fail(cuda_fail(cudaGetLastError(), "reading entry count"));
                nnz = (int64_t)last_pos + last_head;
                if (cudaMalloc(&g->colidx, sizeof(int32_t) * (size_t)(nnz + kCsrPad)) != cudaSuccess ||
                    cudaMalloc(&g->val, sizeof(float) * (size_t)(nnz + kCsrPad)) != cudaSuccess) {
                    cudaGetLastError();
                    set_error("device allocation failed for %lld entries", (long long)nnz);
                    return fail(SF_ERR_OOM);
                }
                compact_runs_kernel<<<(unsigned)((valid + 255) / 256), 256, 0, s>>>(
                    k0, v0, head, pos, valid, cb, g->colidx, g->val, rowcnt);
                if ((st = check_launch("compact_runs_kernel"))) return fail(st);
            }
        }
        g->nnz = nnz;
        if (!g->colidx) {
            if (cudaMalloc(&g->colidx, sizeof(int32_t) * kCsrPad) != cudaSuccess ||
                cudaMalloc(&g->val, sizeof(float) * kCsrPad) != cudaSuccess) {
                cudaGetLastError();
                set_error("device allocation failed");
                return fail(SF_ERR_OOM);
            }
        }
        if (cudaMemsetAsync(g->colidx + nnz, 0, sizeof(int32_t) * kCsrPad, s) != cudaSuccess ||
            cudaMemsetAsync(g->val + nnz, 0, sizeof(float) * kCsrPad, s) != cudaSuccess)
            return fail(cuda_fail(cudaGetLastError(), "cudaMemsetAsync"));
        if ((st = exclusive_scan_i32(rowcnt, g->rowptr, (int64_t)n_nodes + 1, s))) return fail(st);
        fill_i32_kernel<<<1, 32, 0, s>>>(g->rowptr + n_nodes + 1, kCsrPad, (int32_t)nnz);
        if ((st = check_launch("fill_i32_kernel"))) return fail(st);
        if ((st = compute_strength(g, s))) return fail(st);
    }
    *out = g;
    return SF_OK;
}

SF_API sf_status sf_graph_info(const sf_graph *g, int32_t *n, int64_t *nnz_off, int32_t *unit_weights,
                               double *max_strength) {
    SF_ARG(g, "graph is NULL");
    if (n) *n = g->n;
    if (nnz_off) *nnz_off = g->nnz;
    if (unit_weights) *unit_weights = g->unit_weights;
    if (max_strength) *max_strength = g->max_strength;
    return SF_OK;
}

SF_API sf_status sf_graph_csr(const sf_graph *g, const int32_t **rowptr, const int32_t **colidx,
                              const float **val, const double **strength) {
    SF_ARG(g, "graph is NULL");
    if (rowptr) *rowptr = g->rowptr;
    if (colidx) *colidx = g->colidx;
    if (val) *val = g->val;
    if (strength) *strength = g->strength;
    return SF_OK;
}

SF_API sf_status sf_graph_normalize(const sf_graph *g, void *stream, sf_graph **out) {
    SF_ARG(g && out, "graph/out is NULL");
    SF_ARG(!g->normalized, "the graph is already normalised");
    SF_ARG(g->device == current_device(), "graph lives on another device");
    cudaStream_t s = (cudaStream_t)stream;
    sf_graph *h = new sf_graph();
    h->n = g->n;
    h->nnz = g->nnz;
    h->unit_weights = 0;
    h->normalized = 1;
    h->device = g->device;
    auto fail = [&](sf_status e) {
        graph_release(h);
        return e;
    };
    const size_t nz = (size_t)g->nnz + kCsrPad;
    if (cudaMalloc(&h->rowptr, sizeof(int32_t) * (size_t)(g->n + 1 + kCsrPad)) != cudaSuccess ||
        cudaMalloc(&h->colidx, sizeof(int32_t) * nz) != cudaSuccess ||
        cudaMalloc(&h->val, sizeof(float) * nz) != cudaSuccess ||
        cudaMalloc(&h->strength, sizeof(double) * (size_t)g->n) != cudaSuccess) {
        cudaGetLastError();
        set_error("device allocation failed for the normalised graph");
        return fail(SF_ERR_OOM);
    }
    sf_status st;
    Scratch sc(s);
    int32_t *any = nullptr;
    if ((st = sc.get(&any, 1))) return fail(st);
    if (cudaMemcpyAsync(h->rowptr, g->rowptr, sizeof(int32_t) * (size_t)(g->n + 1 + kCsrPad),
                        cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(h->colidx, g->colidx, sizeof(int32_t) * nz, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(h->val, 0, sizeof(float) * nz, s) != cudaSuccess ||
        cudaMemsetAsync(any, 0, sizeof(int32_t), s) != cudaSuccess)
        return fail(cuda_fail(cudaGetLastError(), "copying the pattern"));
    normalize_kernel<<<(g->n + 255) / 256, 256, 0, s>>>(g->n, g->rowptr, g->colidx, g->unit_weights ? nullptr : g->val,
                                                        g->strength, h->val, h->strength, any);
    if ((st = check_launch("normalize_kernel"))) return fail(st);
    int32_t hany = 0;
    if (cudaMemcpyAsync(&hany, any, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail(cuda_fail(cudaGetLastError(), "reading the normalised graph"));
    h->max_strength = hany ? 1.0 : 0.0;
    *out = h;
    return SF_OK;
}

SF_API sf_status sf_graph_set_values(sf_graph *g, const float *val, void *stream) {
    SF_ARG(g, "graph is NULL");
    SF_ARG(!g->normalized, "a normalised graph keeps the weights it was built with (normalise the new weights)");
    SF_ARG(g->nnz == 0 || val, "val is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    if (g->nnz > 0)
        SF_CHECK_CUDA(cudaMemcpyAsync(g->val, val, sizeof(float) * (size_t)g->nnz, cudaMemcpyDeviceToDevice, s));
    {
        // the sliced-ELL copy holds the old weights: rebuild it on next use
        std::lock_guard<std::mutex> lk(g->sell_mu);
        SF_CHECK_CUDA(cudaStreamSynchronize(s));
        sell_release(&g->sell);
    }
    return compute_strength(g, s);
}

SF_API void sf_graph_free(sf_graph *g) {
    if (g) cudaDeviceSynchronize();
    graph_release(g);
}

}  // extern "C"

// ---------------------------------------------------------------- batches
namespace sf {

__global__ void batch_copy_rows_kernel(const int32_t *rowptr, int32_t n, int32_t row_off, int32_t nnz_off,
                                       int32_t gid, const double *strength, int32_t *rowptr_out,
                                       double *strength_out, int32_t *row_graph) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    rowptr_out[row_off + i] = rowptr[i] + nnz_off;
    strength_out[row_off + i] = strength[i];
    row_graph[row_off + i] = gid;
}

__global__ void batch_copy_entries_kernel(const int32_t *colidx, const float *val, int64_t nnz, int32_t row_off,
                                          int64_t nnz_off, int32_t *colidx_out, float *val_out) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    colidx_out[nnz_off + e] = colidx[e] + row_off;
    val_out[nnz_off + e] = val[e];
}

static void batch_release(sf_batch *b) {
    if (!b) return;
    sell_release(&b->sell);
    cudaFree(b->rowptr);
    cudaFree(b->colidx);
    cudaFree(b->val);
    cudaFree(b->strength);
    cudaFree(b->row_graph);
    delete b;
}

}  // namespace sf

extern "C" {

SF_API sf_status sf_batch_build(const sf_graph *const *graphs, int32_t n_graphs, void *stream, sf_batch **out) {
    SF_ARG(out, "out is NULL");
    *out = nullptr;
    SF_ARG(graphs && n_graphs >= 1, "need at least one graph");
    cudaStream_t s = (cudaStream_t)stream;
    sf_batch *b = new sf_batch();
    b->n_graphs = n_graphs;
    b->device = current_device();
    b->offsets.assign((size_t)n_graphs + 1, 0);
    b->nnz_offsets.assign((size_t)n_graphs + 1, 0);
    int64_t n_tot = 0, nnz_tot = 0;
    int unit = 1;
    for (int g = 0; g < n_graphs; ++g) {
        if (!graphs[g]) {
            delete b;
            set_error("graph %d is NULL", g);
            return SF_ERR_ARG;
        }
        n_tot += graphs[g]->n;
        nnz_tot += graphs[g]->nnz;
        unit &= graphs[g]->unit_weights;
        if (n_tot >= INT32_MAX || nnz_tot >= INT32_MAX) {
            delete b;
            set_error("batch too large for int32 indices");
            return SF_ERR_ARG;
        }
        b->offsets[g + 1] = (int32_t)n_tot;
        b->nnz_offsets[g + 1] = nnz_tot;
    }
    b->n = (int32_t)n_tot;
    b->nnz = nnz_tot;
    b->unit_weights = unit;
    if (cudaMalloc(&b->rowptr, sizeof(int32_t) * (size_t)(n_tot + 1 + kCsrPad)) != cudaSuccess ||
        cudaMalloc(&b->strength, sizeof(double) * (size_t)n_tot) != cudaSuccess ||
        cudaMalloc(&b->row_graph, sizeof(int32_t) * (size_t)n_tot) != cudaSuccess ||
        cudaMalloc(&b->colidx, sizeof(int32_t) * (size_t)(nnz_tot + kCsrPad)) != cudaSuccess ||
        cudaMalloc(&b->val, sizeof(float) * (size_t)(nnz_tot + kCsrPad)) != cudaSuccess) {
        cudaGetLastError();
        batch_release(b);
        set_error("device allocation failed for a batch of %lld rows", (long long)n_tot);
        return SF_ERR_OOM;
    }
    sf_status st;
    for (int g = 0; g < n_graphs; ++g) {
        const sf_graph *G = graphs[g];
        batch_copy_rows_kernel<<<(G->n + 255) / 256, 256, 0, s>>>(G->rowptr, G->n, b->offsets[g],
                                                                   (int32_t)b->nnz_offsets[g], g, G->strength,
                                                                   b->rowptr, b->strength, b->row_graph);
        if ((st = check_launch("batch_copy_rows_kernel"))) {
            batch_release(b);
            return st;
        }
        if (G->nnz > 0) {
            batch_copy_entries_kernel<<<(unsigned)((G->nnz + 255) / 256), 256, 0, s>>>(
                G->colidx, G->val, G->nnz, b->offsets[g], b->nnz_offsets[g], b->colidx, b->val);
            if ((st = check_launch("batch_copy_entries_kernel"))) {
                batch_release(b);
                return st;
            }
        }
    }
    fill_i32_kernel<<<1, 32, 0, s>>>(b->rowptr + n_tot, kCsrPad + 1, (int32_t)nnz_tot);
    if ((st = check_launch("fill_i32_kernel"))) {
        batch_release(b);
        return st;
    }
    if (cudaMemsetAsync(b->colidx + nnz_tot, 0, sizeof(int32_t) * kCsrPad, s) != cudaSuccess ||
        cudaMemsetAsync(b->val + nnz_tot, 0, sizeof(float) * kCsrPad, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        st = cuda_fail(cudaGetLastError(), "finishing batch");
        batch_release(b);
        return st;
    }
    *out = b;
    return SF_OK;
}

SF_API sf_status sf_batch_info(const sf_batch *b, int32_t *n_total, int64_t *nnz_total, int32_t *n_graphs,
                               int32_t *row_offsets) {
    SF_ARG(b, "batch is NULL");
    if (n_total) *n_total = b->n;
    if (nnz_total) *nnz_total = b->nnz;
    if (n_graphs) *n_graphs = b->n_graphs;
    if (row_offsets)
        for (int g = 0; g <= b->n_graphs; ++g) row_offsets[g] = b->offsets[g];
    return SF_OK;
}

SF_API void sf_batch_free(sf_batch *b) {
    if (b) cudaDeviceSynchronize();
    batch_release(b);
}

}  // extern "C"
