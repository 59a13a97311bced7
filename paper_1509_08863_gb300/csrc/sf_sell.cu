// Sliced-ELL copy of a CSR for the sweep kernels.
//
// Rows are sorted by decreasing length (ties by index) inside windows of
// 2^kSellWindowLog2 consecutive rows, then cut into slices of kSliceRows
// rows. A slice is padded to the length of its longest row rounded up to a
// multiple of 4 and stored row after row; padding entries carry index n (a
// zero row appended to every gathered block) and weight 0. Slice offsets are
// therefore multiples of 32 entries (128 bytes) and every row starts on a
// 16-byte boundary. The slice count is padded to a multiple of
// kSellSliceAlign with empty slices so that whole tiles can be bulk-copied.
// The window is about as many rows as the sweep kernels process at once, so
// the sort keeps whatever locality the row order has at that scale while the
// slices of one tile (64 or 128 consecutive sorted rows) have nearly equal
// lengths: the warps of a tile finish together and padding stays small.
// Every step is deterministic (stable radix sort, max, prefix sum, copy).
#include "sf_step.cuh"

namespace sf {

constexpr int kSellWindowLog2 = 15;
constexpr int kSellSliceAlign = 16;

// key = window (bits 48..63) | 0xffff - min(length, 0xffff) (bits 32..47) | row (bits 0..31);
// a stable sort on bits 32..63 orders rows by window, then length descending, then index.
__global__ void sell_key_kernel(int32_t n, const int32_t *rowptr, uint64_t *keys) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t len = (uint32_t)min(rowptr[i + 1] - rowptr[i], 0xffff);
    keys[i] = ((uint64_t)((uint32_t)i >> kSellWindowLog2) << 48) | ((uint64_t)(0xffffu - len) << 32) | (uint32_t)i;
}

__global__ void sell_perm_kernel(int32_t n, const uint64_t *keys, int32_t *perm) {
    const int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) perm[t] = (int32_t)(uint32_t)(keys[t] & 0xffffffffull);
}

// entries of slice s = 8 * (longest row length rounded up to 4)
__global__ void sell_slice_len_kernel(int32_t n_slices, const int32_t *rowptr, const int32_t *perm,
                                      int32_t *slen) {
    const int32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_slices) return;
    int32_t mx = 0;
    for (int k = 0; k < kSliceRows; ++k) {
        const int32_t r = perm[(int64_t)s * kSliceRows + k];
        if (r >= 0) mx = max(mx, rowptr[r + 1] - rowptr[r]);
    }
    slen[s] = kSliceRows * ((mx + 3) & ~3);
}

// One thread per slice row: copy the row's entries, pad with (n, 0).
__global__ void sell_fill_kernel(int32_t n, int32_t n_slices, const int32_t *rowptr, const int32_t *colidx,
                                 const float *val, const int32_t *perm, const int32_t *sptr, int32_t *idx,
                                 float *sval) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n_slices * kSliceRows) return;
    const int32_t s = (int32_t)(t / kSliceRows), pos = (int32_t)(t % kSliceRows);
    const int32_t so = sptr[s], ls = (sptr[s + 1] - so) / kSliceRows;
    const int32_t r = perm[t];
    const int32_t beg = r >= 0 ? rowptr[r] : 0, len = r >= 0 ? rowptr[r + 1] - beg : 0;
    int32_t *ip = idx + so + (int64_t)pos * ls;
    float *wp = sval ? sval + so + (int64_t)pos * ls : nullptr;
    for (int32_t j = 0; j < ls; ++j) {
        const bool real = j < len;
        ip[j] = real ? colidx[beg + j] : n;
        if (wp) wp[j] = real ? val[beg + j] : 0.0f;
    }
}

// iperm[perm[t]] = t for every slice row t holding a row
__global__ void sell_iperm_kernel(int64_t count, const int32_t *perm, int32_t *iperm) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < count && perm[t] >= 0) iperm[perm[t]] = (int32_t)t;
}

// ridx[e] = slice row of idx[e] (padding index n becomes the zero row `rows`)
__global__ void sell_renumber_kernel(int64_t count, int32_t n, int32_t rows, const int32_t *idx,
                                     const int32_t *iperm, int32_t *ridx) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= count) return;
    const int32_t k = idx[e];
    ridx[e] = (k >= 0 && k < n) ? iperm[k] : rows;
}

__global__ void sell_fill_pad_kernel(int32_t *p, int count, int32_t v) {
    if ((int)threadIdx.x < count) p[threadIdx.x] = v;
}

void sell_release(SellMatrix *S) {
    cudaFree(S->sptr);
    cudaFree(S->iperm);
    cudaFree(S->perm);
    cudaFree(S->idx);
    cudaFree(S->ridx);
    cudaFree(S->val);
    *S = SellMatrix();
}

sf_status sell_build(SellMatrix *S, int32_t n, const int32_t *rowptr, const int32_t *colidx, const float *val,
                     cudaStream_t s) {
    if (S->built) return SF_OK;
    sell_release(S);
    int32_t n_slices = (n + kSliceRows - 1) / kSliceRows;
    n_slices = (n_slices + kSellSliceAlign - 1) / kSellSliceAlign * kSellSliceAlign;
    const int64_t perm_len = (int64_t)n_slices * kSliceRows;
    sf_status st;
    auto oom = [&]() {
        cudaGetLastError();
        sell_release(S);
        set_error("device allocation failed for the sliced-ELL copy");
        return SF_ERR_OOM;
    };
    if (cudaMalloc(&S->perm, sizeof(int32_t) * (size_t)perm_len) != cudaSuccess ||
        cudaMalloc(&S->sptr, sizeof(int32_t) * (size_t)(n_slices + 1 + kCsrPad)) != cudaSuccess)
        return oom();
    SF_CHECK_CUDA(cudaMemsetAsync(S->perm, 0xff, sizeof(int32_t) * (size_t)perm_len, s));  // -1
    if (n > 0) {
        Scratch sc(s);
        uint64_t *keys = nullptr, *keys_alt = nullptr;
        float *no_vals = nullptr, *no_vals_alt = nullptr;
        if ((st = sc.get(&keys, (size_t)n)) || (st = sc.get(&keys_alt, (size_t)n))) return st;
        sell_key_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, rowptr, keys);
        if ((st = check_launch("sell_key_kernel"))) return st;
        if ((st = radix_sort(keys, no_vals, keys_alt, no_vals_alt, n, 32, 64, s))) return st;
        sell_perm_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, keys, S->perm);
        if ((st = check_launch("sell_perm_kernel"))) return st;
    }
    {
        Scratch sc(s);
        int32_t *slen = nullptr;
        if ((st = sc.get(&slen, (size_t)n_slices + 1))) return st;
        sell_slice_len_kernel<<<(n_slices + 255) / 256, 256, 0, s>>>(n_slices, rowptr, S->perm, slen);
        if ((st = check_launch("sell_slice_len_kernel"))) return st;
        SF_CHECK_CUDA(cudaMemsetAsync(slen + n_slices, 0, sizeof(int32_t), s));
        if ((st = exclusive_scan_i32(slen, S->sptr, (int64_t)n_slices + 1, s))) return st;
    }
    int32_t total = 0;
    SF_CHECK_CUDA(cudaMemcpyAsync(&total, S->sptr + n_slices, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    SF_CHECK_CUDA(cudaStreamSynchronize(s));
    sell_fill_pad_kernel<<<1, 32, 0, s>>>(S->sptr + n_slices + 1, kCsrPad, total);
    if ((st = check_launch("sell_fill_pad_kernel"))) return st;
    if (cudaMalloc(&S->idx, sizeof(int32_t) * (size_t)(total + kCsrPad)) != cudaSuccess) return oom();
    if (val && cudaMalloc(&S->val, sizeof(float) * (size_t)(total + kCsrPad)) != cudaSuccess) return oom();
    const int64_t threads = (int64_t)n_slices * kSliceRows;
    sell_fill_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(n, n_slices, rowptr, colidx, val, S->perm,
                                                                       S->sptr, S->idx, S->val);
    if ((st = check_launch("sell_fill_kernel"))) return st;
    if (cudaMalloc(&S->iperm, sizeof(int32_t) * (size_t)(n > 0 ? n : 1)) != cudaSuccess) return oom();
    sell_iperm_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(threads, S->perm, S->iperm);
    if ((st = check_launch("sell_iperm_kernel"))) return st;
    // the sweeps' copy of the indices, renumbered into slice-row order
    const int32_t rows = n_slices * kSliceRows;
    if (cudaMalloc(&S->ridx, sizeof(int32_t) * (size_t)(total + kCsrPad)) != cudaSuccess) return oom();
    if (total > 0) {
        sell_renumber_kernel<<<(unsigned)(((int64_t)total + 255) / 256), 256, 0, s>>>(total, n, rows, S->idx,
                                                                                        S->iperm, S->ridx);
        if ((st = check_launch("sell_renumber_kernel"))) return st;
    }
    sell_fill_pad_kernel<<<1, 32, 0, s>>>(S->ridx + total, kCsrPad, rows);
    if ((st = check_launch("sell_fill_pad_kernel"))) return st;
    S->n = n;
    S->n_slices = n_slices;
    S->rows = rows;
    S->entries = total;
    S->built = true;
    return SF_OK;
}

}  // namespace sf
