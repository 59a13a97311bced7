// The persistent batch sweep: every order of a batch of graphs in one launch
// (cheb_batch_kernel in sf_step.cuh), with per-graph arrival counters so that
// each graph advances to its next order as soon as its own tiles are done.
#include "sf_step.cuh"

namespace sf {

using BatchFn = void (*)(const StepParams, const BatchSched);

template <typename TS, int LPR, bool W>
static BatchFn batch_fn_mode(int mode) {
    return mode == MODE_FWD ? cheb_batch_kernel<TS, LPR, MODE_FWD, W> : cheb_batch_kernel<TS, LPR, MODE_CLEN, W>;
}

template <typename TS, bool W>
static BatchFn batch_fn_lpr(int lpr, int mode) {
    switch (lpr) {
        case 2: return batch_fn_mode<TS, 2, W>(mode);
        case 4: return batch_fn_mode<TS, 4, W>(mode);
        case 8: return batch_fn_mode<TS, 8, W>(mode);
        case 16: return batch_fn_mode<TS, 16, W>(mode);
        case 32: return batch_fn_mode<TS, 32, W>(mode);
        default: return nullptr;
    }
}

static BatchFn batch_fn(int storage, int lpr, int mode, bool weighted) {
    if (mode != MODE_FWD && mode != MODE_CLEN) return nullptr;
    if (storage == SF_F32) return weighted ? batch_fn_lpr<float, true>(lpr, mode) : batch_fn_lpr<float, false>(lpr, mode);
    if (storage == SF_BF16)
        return weighted ? batch_fn_lpr<__nv_bfloat16, true>(lpr, mode) : batch_fn_lpr<__nv_bfloat16, false>(lpr, mode);
    if (storage == SF_F16)
        return weighted ? batch_fn_lpr<__half, true>(lpr, mode) : batch_fn_lpr<__half, false>(lpr, mode);
    return nullptr;
}

static int batch_rows_per_tile(int lpr) { return lpr == 2 ? TileCfg<2>::rows : TileCfg<4>::rows; }

static int batch_smem(int lpr, bool weighted) {
    switch (lpr) {
        case 2: return TileCfg<2>::smem_bytes(weighted);
        case 4: return TileCfg<4>::smem_bytes(weighted);
        case 8: return TileCfg<8>::smem_bytes(weighted);
        case 16: return TileCfg<16>::smem_bytes(weighted);
        default: return TileCfg<32>::smem_bytes(weighted);
    }
}

// Per chunk (rows_per_chunk consecutive slice rows): the range of graph ids
// among its rows; per graph: the number of chunks whose range covers it (the
// arrival count that completes one order).
__global__ void chunk_range_kernel(int32_t n, int64_t rows_per_chunk, int32_t n_chunks, const int32_t *gid_t,
                                   int32_t *glo, int32_t *ghi, uint32_t *graph_chunks) {
    const int32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_chunks) return;
    const int64_t r0 = (int64_t)c * rows_per_chunk;
    const int64_t r1 = r0 + rows_per_chunk < n ? r0 + rows_per_chunk : n;
    int32_t lo = gid_t[r0], hi = lo;
    for (int64_t r = r0 + 1; r < r1; ++r) {
        lo = min(lo, gid_t[r]);
        hi = max(hi, gid_t[r]);
    }
    glo[c] = lo;
    ghi[c] = hi;
    for (int32_t g = lo; g <= hi; ++g) atomicAdd(graph_chunks + g, 1u);
}

sf_status make_batch_shape(int storage, int slab_cols, int block_warps, int blocks_per_sm, int mode, bool weighted,
                           int carveout_pct, SweepShape *sh) {
    sf_status st = make_shape(storage, slab_cols, block_warps, blocks_per_sm, mode, weighted, sh, carveout_pct,
                              SF_SWEEP_TILED);
    if (st) return st;
    const BatchFn fn = batch_fn(storage, sh->lpr, mode, weighted);
    SF_ARG(fn, "no persistent batch kernel for this shape");
    const int smem = batch_smem(sh->lpr, weighted);
    SF_CHECK_CUDA(cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    SF_CHECK_CUDA(cudaFuncSetAttribute((const void *)fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                       carveout_pct > 0 ? carveout_pct : cudaSharedmemCarveoutDefault));
    int occ = 0;
    SF_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void *)fn, sh->block, smem));
    if (occ < 1) occ = 1;
    if (blocks_per_sm > 0 && blocks_per_sm < occ) occ = blocks_per_sm;
    sh->grid = occ * sm_count();  // co-resident blocks (the queue needs no more)
    sh->smem = smem;
    sh->direct = false;
    return SF_OK;
}

sf_status launch_batch_persistent(const SweepShape &sh, int mode, StepParams P, int32_t n_graphs, int32_t p,
                                  const int32_t *gid_t, void *const buf[3], cudaStream_t s, double bytes) {
    const BatchFn fn = batch_fn(sh.storage, sh.lpr, mode, sh.weighted);
    SF_ARG(fn, "no persistent batch kernel for this shape");
    SF_ARG(gid_t && n_graphs >= 1 && p >= 1, "persistent batch sweep needs graph ids, graphs and p >= 1");
    const int rpt = batch_rows_per_tile(sh.lpr);
    const int32_t n_tiles = (P.n + rpt - 1) / rpt;
    if (n_tiles == 0) return SF_OK;
    // tiles per item: up to kBatchChunk, fewer when a step has too few tiles to give every resident block
    // two items (an item's latency, not the work, would then set the time of a step); at one or two tiles
    // the claim and the counter polls cost more than they save (a 256-graph batch of 300-2500 nodes: 10.1,
    // 8.6, 8.0 and 12.9 ms at 1, 2, 4 and 8 tiles per item)
    int32_t chunk = n_tiles / (2 * sh.grid);
    chunk = chunk < 1 ? 1 : (chunk > kBatchChunk ? kBatchChunk : chunk);
    const int32_t n_chunks = (n_tiles + chunk - 1) / chunk;
    SF_ARG((int64_t)n_chunks * p < (1ll << 31), "batch too large for 32-bit work items (chunks x orders)");
    Scratch sc(s);
    int32_t *glo = nullptr, *ghi = nullptr, *abort = nullptr;
    uint32_t *graph_chunks = nullptr, *done = nullptr, *queue = nullptr;
    sf_status st;
    if ((st = sc.get(&glo, (size_t)n_chunks)) || (st = sc.get(&ghi, (size_t)n_chunks)) ||
        (st = sc.get(&graph_chunks, (size_t)n_graphs)) || (st = sc.get(&done, (size_t)n_graphs)) ||
        (st = sc.get(&queue, 1)) || (st = sc.get(&abort, 1)))
        return st;
    SF_CHECK_CUDA(cudaMemsetAsync(graph_chunks, 0, sizeof(uint32_t) * (size_t)n_graphs, s));
    SF_CHECK_CUDA(cudaMemsetAsync(done, 0, sizeof(uint32_t) * (size_t)n_graphs, s));
    SF_CHECK_CUDA(cudaMemsetAsync(queue, 0, sizeof(uint32_t), s));
    SF_CHECK_CUDA(cudaMemsetAsync(abort, 0, sizeof(int32_t), s));
    chunk_range_kernel<<<(unsigned)((n_chunks + 255) / 256), 256, 0, s>>>(P.n, (int64_t)rpt * chunk, n_chunks, gid_t,
                                                                        glo, ghi, graph_chunks);
    if ((st = check_launch("chunk_range_kernel"))) return st;
    BatchSched S = {};
    S.n_tiles = n_tiles;
    S.chunk = chunk;
    S.n_chunks = n_chunks;
    S.p = p;
    S.chunk_glo = glo;
    S.chunk_ghi = ghi;
    S.graph_chunks = graph_chunks;
    S.done = done;
    S.queue = queue;
    S.abort = abort;
    for (int k = 0; k < 3; ++k) S.buf[k] = buf[k];
    cudaEvent_t ea = nullptr, eb = nullptr;
    const bool prof = profiling_on() && !profile_span_active() && profile_events(&ea, &eb);
    if (prof) cudaEventRecord(ea, s);
    fn<<<sh.grid, sh.block, sh.smem, s>>>(P, S);
    st = check_launch("cheb_batch_kernel");
    if (prof) {
        cudaEventRecord(eb, s);
        profile_record(ea, eb, bytes, mode * 3 + sh.storage);
    }
    return st;
}

}  // namespace sf
