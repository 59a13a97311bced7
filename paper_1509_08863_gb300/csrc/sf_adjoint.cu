// Adjoint of the filter Y = sum_j a_j T_j(Lt) R for the loss l = <G, Y>.
//
// Reverse mode of the three-term recurrence (Lt is symmetric):
//   Gb_p = a_p G;  Gb_j = a_j G + 2 Lt Gb_{j+1} - Gb_{j+2} (1 <= j < p);
//   Gb_0 = a_0 G + Lt Gb_1 - Gb_2 = dl/dR;
//   dl/da_j = <G, T_j R>;
//   M = dl/dLt on the stored pattern and the diagonal
//     = Gb_1 T_0^T + sum_{j >= 2} 2 Gb_j T_{j-1}^T   (a sampled dense-dense
//       product: only entries (u, v) with W_uv stored, plus (u, u));
//   dl/dW_uv = (2/lam)(M_uu + M_vv - M_uv - M_vu) (L = S - W, §2.1).
// Per order: Gb_j is one Clenshaw sweep (the sweep kernel with G as the
// addend block); the sampled products and <G, T_j> are a second kernel that
// walks the same sliced-ELL tiles (TMA-staged) and gathers rows of T_{j-1}.
// The edge accumulators are kept in sliced-ELL order and mapped back to CSR
// order once at the end.
#include <math.h>

#include "sf_step.cuh"

namespace sf {

// Blocks are in slice-row order (row t of a block is graph row perm[t], see
// SellMatrix); sell_idx holds the column indices as slice rows.
struct SddmmParams {
    int32_t n;
    int64_t sell_slices;
    const int32_t *sell_ptr;
    const int32_t *sell_idx;
    int32_t ld;
    const float *Gb;   // Gb_j, own rows
    const float *Tm1;  // T_{j-1}: gathered for the sampled products, own row for the diagonal (nullptr: none)
    const float *Gq;   // packed G, own rows
    const float *Tj;   // T_j own rows, for <G, T_j>
    float csd;         // 1 for j == 1, 2 for j >= 2
    float *Msell;      // [entries] accumulated edge products, sliced-ELL order
    float *Mdiag;      // [rows] accumulated diagonal products, slice-row order
    double *part;      // [gridDim.x] partial <G, T_j>
    int32_t *status;
};

// sum of v over the LPR lanes of a group (all lanes get the sum); `mask` holds
// the group's lanes only, so groups of one warp may diverge (padding rows,
// slices of different lengths)
template <int LPR>
__device__ __forceinline__ float group_sum(unsigned mask, float v) {
#pragma unroll
    for (int off = 1; off < LPR; off <<= 1) v += __shfl_xor_sync(mask, v, off);
    return v;
}

__device__ __forceinline__ float dot4(const float4 a, const float4 b) {
    return fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, a.w * b.w)));
}

template <int LPR>
__global__ void __launch_bounds__(256, 4) sddmm_kernel(const SddmmParams P) {
    using C = TileCfg<LPR>;
    constexpr int VEC = 4;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t *s_bar = reinterpret_cast<uint64_t *>(smem_raw);      // [2]
    int32_t *s_meta = reinterpret_cast<int32_t *>(smem_raw + 16);  // [2][2]: entry base, fits
    unsigned char *s_buf0 = smem_raw + C::header;
    constexpr int buf_bytes = C::buf_bytes(false);
    static_assert(C::stages >= 2, "two stage buffers");
    __shared__ double s_red[8];

    const int tid = threadIdx.x;
    const int q = tid % LPR, grp = tid / LPR;
    const int ngrp = blockDim.x / LPR;
    const int n_tiles = (P.n + C::rows - 1) / C::rows;
    const int32_t ld = P.ld;
    const unsigned gmask = (LPR == 32) ? 0xffffffffu : (((1u << LPR) - 1u) << ((tid & 31) & ~(LPR - 1)));
    const float *__restrict__ Tm1q = P.Tm1 ? P.Tm1 + q * VEC : nullptr;
    double gdot = 0.0;

    auto issue = [&](int tile, int b) {
        unsigned char *base = s_buf0 + b * buf_bytes;
        int32_t *sp = reinterpret_cast<int32_t *>(base);
        int32_t *ix = sp + C::sp_ints;
        const int32_t s0 = tile * C::slices;
        const int32_t e0 = P.sell_ptr[s0], e1 = P.sell_ptr[s0 + C::slices];
        const int32_t cnt = e1 - e0;
        const bool fits = (P.Tm1 != nullptr) && cnt <= C::entries;
        const uint32_t bytes = C::sp_ints * 4 + (fits ? (uint32_t)cnt * 4u : 0u);
        s_meta[2 * b] = e0;
        s_meta[2 * b + 1] = fits ? 1 : 0;
        fence_proxy_async();
        mbar_arrive_expect_tx(&s_bar[b], bytes);
        bulk_g2s(sp, P.sell_ptr + s0, C::sp_ints * 4, &s_bar[b]);
        if (fits && cnt > 0) bulk_g2s(ix, P.sell_idx + e0, cnt * 4, &s_bar[b]);
    };

    if (tid == 0) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        fence_mbar_init();
        if ((int)blockIdx.x < n_tiles) issue(blockIdx.x, 0);
    }
    __syncthreads();
    for (int k = 0;; ++k) {
        const int tile = blockIdx.x + k * gridDim.x;
        if (tile >= n_tiles) break;
        const int b = k & 1;
        if (tid == 0 && tile + (int)gridDim.x < n_tiles) issue(tile + gridDim.x, b ^ 1);
        const bool landed = mbar_wait_bounded(&s_bar[b], (uint32_t)(k >> 1) & 1u);
        if (__syncthreads_or(!landed)) {
            if (tid == 0) atomicOr(P.status, 1);
            mbar_wait_bounded(&s_bar[b], (uint32_t)(k >> 1) & 1u);
            if (tile + (int)gridDim.x < n_tiles) mbar_wait_bounded(&s_bar[b ^ 1], (uint32_t)((k + 1) >> 1) & 1u);
            return;
        }
        const int32_t *s_sp = reinterpret_cast<const int32_t *>(s_buf0 + b * buf_bytes);
        const int32_t *s_ix = s_sp + C::sp_ints;
        const int32_t e0 = s_meta[2 * b];
        const bool fits = s_meta[2 * b + 1] != 0;

        for (int tr = grp; tr < C::rows; tr += ngrp) {
            const int32_t i = tile * C::rows + tr;  // slice row: the row of every block
            if (i >= P.n) continue;
            const int sl = tr / kSliceRows, pos = tr % kSliceRows;
            const int32_t so = s_sp[sl], ls = (s_sp[sl + 1] - so) / kSliceRows;
            const int32_t eo = so - e0 + pos * ls;
            const int64_t ro = (int64_t)i * ld + q * VEC;
            if (P.Tj) {
                const float4 gq = __ldg(reinterpret_cast<const float4 *>(P.Gq + ro));
                const float4 tj = __ldg(reinterpret_cast<const float4 *>(P.Tj + ro));
                const float s = group_sum<LPR>(gmask, dot4(gq, tj));
                if (q == 0) gdot += (double)s;
            }
            if (!P.Tm1) continue;
            const float4 gb = __ldg(reinterpret_cast<const float4 *>(P.Gb + ro));
            {
                const float4 tp = __ldg(reinterpret_cast<const float4 *>(P.Tm1 + ro));
                const float s = group_sum<LPR>(gmask, dot4(gb, tp));
                if (q == 0) P.Mdiag[i] += P.csd * s;
            }
            const int32_t *ip = fits ? s_ix + eo : P.sell_idx + e0 + eo;
            float *mp = P.Msell + (int64_t)e0 + eo;  // 16-byte aligned: rows start on multiples of 4
            // eight entries per pass (four in the last one when ls is not a multiple of 8): their gathers and
            // the accumulators they add into are all requested before the first product is reduced
            for (int32_t j = 0; j < ls; j += 8) {
                const bool two = j + 4 < ls;
                const int4 a = fits ? lds_int4(ip + j) : __ldg(reinterpret_cast<const int4 *>(ip + j));
                const int4 b = two ? (fits ? lds_int4(ip + j + 4) : __ldg(reinterpret_cast<const int4 *>(ip + j + 4)))
                                   : a;
                const int32_t kk[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
                if constexpr (LPR >= 8) {
                    // the group's 8 partial sums are reduced transposed: three exchange steps leave lane q
                    // with the sum over LPR / 8 ... of entry q / (LPR / 8), the remaining steps finish it
                    constexpr int kSub = LPR / 8;
                    const int e = q / kSub;
                    const bool writer = q % kSub == 0 && (two || e < 4);
                    const float m = writer ? __ldcg(mp + j + e) : 0.f;
                    float4 x[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        x[u] = __ldg(reinterpret_cast<const float4 *>(Tm1q + (uint32_t)kk[u] * (uint32_t)ld));
                    float d[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) d[u] = dot4(gb, x[u]);
#pragma unroll
                    for (int st = 0; st < 3; ++st) {
                        const int o = LPR >> (st + 1);
                        const int half = 4 >> st;
                        const bool up = (q & o) != 0;
#pragma unroll
                        for (int i = 0; i < half; ++i) {
                            const float send = up ? d[i] : d[i + half];
                            const float keep = up ? d[i + half] : d[i];
                            d[i] = keep + __shfl_xor_sync(gmask, send, o);
                        }
                    }
                    float v = d[0];
#pragma unroll
                    for (int o = kSub / 2; o > 0; o >>= 1) v += __shfl_xor_sync(gmask, v, o);
                    if (writer) mp[j + e] = fmaf(P.csd, v, m);
                } else {
                    float4 m0 = make_float4(0.f, 0.f, 0.f, 0.f), m1 = m0;
                    if (q == 0) {
                        m0 = __ldcg(reinterpret_cast<const float4 *>(mp + j));
                        if (two) m1 = __ldcg(reinterpret_cast<const float4 *>(mp + j + 4));
                    }
                    float4 x[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        x[u] = __ldg(reinterpret_cast<const float4 *>(Tm1q + (uint32_t)kk[u] * (uint32_t)ld));
                    float d[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) d[u] = group_sum<LPR>(gmask, dot4(gb, x[u]));
                    if (q == 0) {
                        m0.x = fmaf(P.csd, d[0], m0.x);
                        m0.y = fmaf(P.csd, d[1], m0.y);
                        m0.z = fmaf(P.csd, d[2], m0.z);
                        m0.w = fmaf(P.csd, d[3], m0.w);
                        *reinterpret_cast<float4 *>(mp + j) = m0;
                        if (two) {
                            m1.x = fmaf(P.csd, d[4], m1.x);
                            m1.y = fmaf(P.csd, d[5], m1.y);
                            m1.z = fmaf(P.csd, d[6], m1.z);
                            m1.w = fmaf(P.csd, d[7], m1.w);
                            *reinterpret_cast<float4 *>(mp + j + 4) = m1;
                        }
                    }
                }
            }
        }
        __syncthreads();  // buffer b fully consumed before it is refilled
    }
    const int w = tid >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) gdot += __shfl_xor_sync(0xffffffffu, gdot, off);
    if ((tid & 31) == 0) s_red[w] = gdot;
    __syncthreads();
    if (tid == 0) {
        double a = 0.0;
        for (int k2 = 0; k2 < (int)(blockDim.x >> 5); ++k2) a += s_red[k2];
        P.part[blockIdx.x] = a;
    }
}

// Position in the sliced-ELL accumulators of the jj-th entry of CSR row u.
__device__ __forceinline__ int64_t sell_pos(const int32_t *sptr, const int32_t *iperm, int32_t u, int32_t jj) {
    const int32_t t = iperm[u];
    const int32_t sl = t / kSliceRows, pos = t % kSliceRows;
    const int32_t so = sptr[sl], ls = (sptr[sl + 1] - so) / kSliceRows;
    return (int64_t)so + (int64_t)pos * ls + jj;
}

// grad[e] = (2/lam)(Md[u] + Md[v] - M_uv - M_vu) for CSR entry e = (u, v); the
// entry (v, u) is found by binary search in the sorted row v. Md is in
// slice-row order.
__global__ void edge_grad_kernel(int32_t n, const int32_t *rowptr, const int32_t *colidx, const int32_t *sptr,
                                 const int32_t *iperm, const float *Msell, const float *Mdiag, float two_over_lam,
                                 float *grad) {
    for (int32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        const int32_t beg = rowptr[u];
        for (int32_t e = beg; e < rowptr[u + 1]; ++e) {
            const int32_t v = colidx[e];
            int32_t lo = rowptr[v], hi = rowptr[v + 1] - 1;
            float mvu = 0.f;
            while (lo <= hi) {
                const int32_t mid = (lo + hi) >> 1;
                const int32_t c = colidx[mid];
                if (c == u) {
                    mvu = Msell[sell_pos(sptr, iperm, v, mid - rowptr[v])];
                    break;
                }
                if (c < u) lo = mid + 1;
                else hi = mid - 1;
            }
            const float muv = Msell[sell_pos(sptr, iperm, u, e - beg)];
            grad[e] = two_over_lam * ((Mdiag[iperm[u]] + Mdiag[iperm[v]]) - (muv + mvu));
        }
    }
}

template <int LPR>
static sf_status sddmm_launch_t(const SddmmParams &P, int grid, int block, cudaStream_t s) {
    const int smem = TileCfg<LPR>::smem_bytes(false);
    cudaError_t e = cudaFuncSetAttribute(sddmm_kernel<LPR>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(sddmm_kernel)");
    sddmm_kernel<LPR><<<grid, block, smem, s>>>(P);
    return check_launch("sddmm_kernel");
}

static sf_status sddmm_launch(int lpr, const SddmmParams &P, int grid, int block, cudaStream_t s, double bytes) {
    cudaEvent_t ea = nullptr, eb = nullptr;
    const bool prof = profiling_on() && profile_events(&ea, &eb);
    if (prof) cudaEventRecord(ea, s);
    sf_status st;
    switch (lpr) {
        case 2: st = sddmm_launch_t<2>(P, grid, block, s); break;
        case 4: st = sddmm_launch_t<4>(P, grid, block, s); break;
        case 8: st = sddmm_launch_t<8>(P, grid, block, s); break;
        case 16: st = sddmm_launch_t<16>(P, grid, block, s); break;
        case 32: st = sddmm_launch_t<32>(P, grid, block, s); break;
        default: set_error("bad lanes per row"); return SF_ERR_ARG;
    }
    if (prof) {
        cudaEventRecord(eb, s);
        profile_record(ea, eb, bytes, kProfTagAdjoint);
    }
    return st;
}

}  // namespace sf

using namespace sf;

extern "C" SF_API sf_status sf_cheb_filter_backward(const sf_graph *g, double lam_max, const double *coeffs,
                                                    int32_t p, const float *R, int32_t n_sig, const float *G,
                                                    float *grad_val, double *grad_coeffs, float *grad_R,
                                                    const sf_opts *opts, void *stream) {
    SF_ARG(g, "graph is NULL");
    SF_ARG(lam_max > 0.0 && isfinite(lam_max), "lam_max must be finite and > 0");
    SF_ARG(p >= 1 && p <= 100000, "p must be in [1, 100000]");
    SF_ARG(n_sig >= 1, "n_sig must be >= 1");
    SF_ARG(coeffs && R && G, "coeffs/R/G is NULL");
    SF_ARG(g->nnz == 0 || grad_val, "grad_val is NULL");
    SF_ARG(g->device == current_device(), "graph lives on another device");
    SF_ARG(!g->normalized, "the adjoint needs L = S - W with S the row sums of W (not a normalised graph)");
    for (int j = 0; j <= p; ++j) SF_ARG(isfinite(coeffs[j]), "coefficient %d is not finite", j);
    sf_opts o = {};
    if (opts) o = *opts;
    SF_ARG(o.storage == SF_F32, "the adjoint keeps FP32 blocks (storage must be SF_F32)");
    if (o.slab_cols <= 0) o.slab_cols = auto_slab_cols(g->n, n_sig, SF_F32, kAutoSlabBudget);
    SweepShape sh;
    sf_status st = make_shape(SF_F32, o.slab_cols, o.block_warps, o.blocks_per_sm, MODE_FWD,
                              !g->unit_weights, &sh, o.carveout_pct, o.sweep_kernel);
    if (st) return st;
    SweepShape shc;  // the Clenshaw sweep kernel of the adjoint (its own attributes and occupancy)
    if ((st = make_shape(SF_F32, o.slab_cols, o.block_warps, o.blocks_per_sm, MODE_CLEN, !g->unit_weights, &shc,
                         o.carveout_pct, o.sweep_kernel)))
        return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = g->n;
    const int ld = sh.ld;
    {
        std::lock_guard<std::mutex> lk(g->sell_mu);
        if ((st = sell_build(&g->sell, g->n, g->rowptr, g->colidx, g->unit_weights ? nullptr : g->val, s))) return st;
    }
    // one block = rows + 1 rows in slice-row order: row `rows` stays zero (padding of the sliced-ELL layout)
    const int64_t rows = g->sell.rows;
    const int32_t *perm = g->sell.perm;
    const size_t blk = (size_t)(rows + 1) * ld;
    SF_ARG((int64_t)(rows + 1) * ld < (1ll << 32), "graph too large for 32-bit slab offsets: use narrower slabs");
    const int64_t cap_mb = o.mem_cap_mb > 0 ? o.mem_cap_mb : 16384;
    int k = o.ckpt_every;
    if (k <= 0) k = ((double)(p + 1) * blk * 4 <= (double)cap_mb * (1 << 20)) ? 1 : (int)ceil(sqrt((double)p));
    if (k > p) k = p;
    // checkpoint slots: 0 and (c-1, c) for c = k, 2k, ... <= p (all j when k == 1)
    std::vector<int> slot((size_t)p + 1, -1);
    int nslots = 0;
    for (int j = 0; j <= p; ++j) {
        if (k == 1 || j == 0 || j % k == 0 || (j + 1) % k == 0) slot[j] = nslots++;
    }
    Scratch sc(s);
    float *store = nullptr, *seg = nullptr, *work[3] = {nullptr, nullptr, nullptr}, *bb[3] = {nullptr, nullptr, nullptr};
    float *gq = nullptr, *coef = nullptr, *dtil = nullptr, *msell = nullptr, *mdiag = nullptr, *gR = nullptr;
    double *part = nullptr, *ga = nullptr;
    if ((st = sc.get(&store, (size_t)nslots * blk))) return st;
    if (k > 1 && (st = sc.get(&seg, (size_t)(k + 1) * blk))) return st;
    for (int q = 0; q < 3; ++q) {
        if ((st = sc.get(&work[q], blk))) return st;
        if ((st = sc.get(&bb[q], blk))) return st;
    }
    if ((st = sc.get(&gq, blk)) || (st = sc.get(&coef, (size_t)p + 1)) || (st = sc.get(&dtil, (size_t)rows)) ||
        (st = sc.get(&mdiag, (size_t)rows)) || (st = sc.get(&part, (size_t)sm_count() * 4 + 1)) ||
        (st = sc.get(&ga, (size_t)p + 1)))
        return st;
    if ((st = sc.get(&msell, (size_t)g->sell.entries + kCsrPad))) return st;
    if (grad_R && (st = sc.get(&gR, blk))) return st;
    SF_CHECK_CUDA(cudaMemsetAsync(store, 0, sizeof(float) * (size_t)nslots * blk, s));
    if (seg) SF_CHECK_CUDA(cudaMemsetAsync(seg, 0, sizeof(float) * (size_t)(k + 1) * blk, s));
    for (int q = 0; q < 3; ++q) {
        SF_CHECK_CUDA(cudaMemsetAsync(work[q], 0, sizeof(float) * blk, s));
        SF_CHECK_CUDA(cudaMemsetAsync(bb[q], 0, sizeof(float) * blk, s));
    }
    {
        std::vector<float> cf((size_t)p + 1);
        for (int j = 0; j <= p; ++j) cf[j] = (float)coeffs[j];
        SF_CHECK_CUDA(cudaMemcpyAsync(coef, cf.data(), sizeof(float) * (p + 1), cudaMemcpyHostToDevice, s));
    }
    SF_CHECK_CUDA(cudaMemsetAsync(msell, 0, sizeof(float) * ((size_t)g->sell.entries + kCsrPad), s));
    SF_CHECK_CUDA(cudaMemsetAsync(mdiag, 0, sizeof(float) * rows, s));
    SF_CHECK_CUDA(cudaMemsetAsync(ga, 0, sizeof(double) * (p + 1), s));
    if (rows > 0) {
        dtil_kernel<<<(unsigned)((rows + 255) / 256), 256, 0, s>>>(g->strength, (int32_t)rows, 2.0 / lam_max, nullptr,
                                                                   nullptr, dtil, nullptr, perm, nullptr);
        if ((st = check_launch("dtil_kernel"))) return st;
    }
    const float *val = g->unit_weights ? nullptr : g->val;
    const int pack_grid = kPackBlocksPerSm * sm_count();
    const double two_over_lam = 2.0 / lam_max;
    const int n_slabs = (n_sig + ld - 1) / ld;

    for (int c0 = 0; c0 < n_sig; c0 += ld) {
        const int w = (n_sig - c0) < ld ? (n_sig - c0) : ld;
        auto T_at = [&](int j) { return store + (size_t)slot[j] * blk; };
        // ---- forward: T_0..T_p, keeping the checkpoint slots
        pack_kernel<float><<<pack_grid, 256, 0, s>>>(R, SF_F32, (int32_t)n, n_sig, c0, w, ld, work[0], nullptr, 0, 0,
                                                     nullptr, 1, 0, nullptr, nullptr, nullptr, nullptr, perm,
                                                     (int32_t)rows);
        if ((st = check_launch("pack_kernel"))) return st;
        SF_CHECK_CUDA(cudaMemcpyAsync(T_at(0), work[0], blk * 4, cudaMemcpyDeviceToDevice, s));
        StepParams P = {};
        P.n = (int32_t)n;
        P.sell_ptr = g->sell.sptr;
        P.sell_idx = g->sell.ridx;
        P.sell_val = g->sell.val;
        P.dtil = dtil;
        P.wscale_u = (float)two_over_lam;
        P.ld = ld;
        P.flags = step_flags(o);
        P.n_cut = 0;
        P.status = device_status();
        // compulsory bytes: the order's CSR once (shared over its slabs), gathered block once,
        // T_{j-2} read, T_j written
        const double csr_b =
            ((double)(n + 1) * 4 + (double)n * 4 + (double)g->nnz * (val ? 8 : 4)) / (double)n_slabs;
        const double blk_b = (double)n * w * 4;
        auto fwd_step = [&](const float *Xp, const float *Zp, float *outp, int j) {
            P.X = Xp;
            P.Z = Zp;
            P.out = outp;
            P.m = (j == 1) ? 1.0f : 2.0f;
            P.j = j;
            return launch_step(sh, MODE_FWD, P, s, csr_b + blk_b * (Zp ? 3 : 2));
        };
        for (int j = 1; j <= p; ++j) {
            float *outp = (k == 1) ? T_at(j) : work[j % 3];
            const float *Xp = (k == 1) ? T_at(j - 1) : work[(j - 1) % 3];
            const float *Zp = (j >= 2) ? ((k == 1) ? T_at(j - 2) : work[(j - 2) % 3]) : nullptr;
            if ((st = fwd_step(Xp, Zp, outp, j))) return st;
            if (k > 1 && slot[j] >= 0)
                SF_CHECK_CUDA(cudaMemcpyAsync(T_at(j), outp, blk * 4, cudaMemcpyDeviceToDevice, s));
        }
        // ---- backward
        int seg_base = -1;
        auto ensure_segment = [&](int jlo) -> sf_status {
            // segment holding T_c .. T_{min(c + k, p)} with c = k * floor(jlo / k)
            const int c = (jlo / k) * k;
            if (c == seg_base) return SF_OK;
            const int top = (c + k < p) ? c + k : p;
            SF_CHECK_CUDA(cudaMemcpyAsync(seg, T_at(c), blk * 4, cudaMemcpyDeviceToDevice, s));
            for (int j = c + 1; j <= top; ++j) {
                const float *Xp = seg + (size_t)(j - 1 - c) * blk;
                const float *Zp = nullptr;
                if (j >= 2) Zp = (j - 2 >= c) ? seg + (size_t)(j - 2 - c) * blk : T_at(j - 2);
                sf_status e = fwd_step(Xp, Zp, seg + (size_t)(j - c) * blk, j);
                if (e) return e;
            }
            seg_base = c;
            return SF_OK;
        };
        auto T_get = [&](int j) -> const float * {
            if (k == 1) return T_at(j);
            if (seg_base >= 0 && j >= seg_base && j <= seg_base + k) return seg + (size_t)(j - seg_base) * blk;
            return T_at(j);  // a checkpoint slot
        };
        // Gb_p = a_p G (pack with b-start), packed G
        pack_kernel<float><<<pack_grid, 256, 0, s>>>(G, SF_F32, (int32_t)n, n_sig, c0, w, ld, gq, nullptr, 0, 1, coef,
                                                     p + 1, p, nullptr, bb[p % 3], nullptr, nullptr, perm,
                                                     (int32_t)rows);
        if ((st = check_launch("pack_kernel"))) return st;
        // the Clenshaw sweep on G: Gb_j = a_j G + m Lt Gb_{j+1} - Gb_{j+2}
        StepParams C = P;
        C.Q = gq;
        C.coef = coef;
        C.coef_ld = p + 1;
        C.n_cut = 1;
        SddmmParams D = {};
        D.n = (int32_t)n;
        D.sell_slices = g->sell.n_slices;
        D.sell_ptr = g->sell.sptr;
        D.sell_idx = g->sell.ridx;
        D.ld = ld;
        D.Gq = gq;
        D.Msell = msell;
        D.Mdiag = mdiag;
        D.part = part;
        D.status = device_status();
        const int sddmm_grid = sm_count() * 4;
        for (int j = p; j >= 0; --j) {
            if (k > 1 && j >= 1 && (st = ensure_segment(j - 1))) return st;
            if (j < p) {
                C.X = bb[(j + 1) % 3];
                C.Z = (j + 2 <= p) ? bb[(j + 2) % 3] : nullptr;
                C.j = j;
                C.m = (j == 0) ? 1.0f : 2.0f;
                C.out = bb[j % 3];
                C.outf = (j == 0) ? (gR ? gR : work[0]) : nullptr;  // dl/dR (scratch target when not requested)
                const double cb = csr_b + blk_b * (C.Z ? 4 : 3);
                if ((st = launch_step(shc, MODE_CLEN, C, s, cb))) return st;
            }
            D.Gb = bb[j % 3];
            D.Tm1 = (j >= 1) ? T_get(j - 1) : nullptr;
            D.Tj = (j >= 1) ? T_get(j) : T_at(0);
            D.csd = (j == 1) ? 1.0f : 2.0f;
            // index stream once, G and T_j rows, Gb_j rows and T_{j-1} gathered once (when products
            // are taken), edge and diagonal accumulators read and written
            const double db = (double)g->sell.entries * 4 / (double)n_slabs + blk_b * 2 +
                              (D.Tm1 ? blk_b * 2 + 8.0 * ((double)g->nnz + n) : 0.0);
            if ((st = sddmm_launch(sh.lpr, D, sddmm_grid, 256, s, db))) return st;
            pair_sum_kernel<<<1, 256, 0, s>>>(part, sddmm_grid, 1, ga + j);
            if ((st = check_launch("pair_sum_kernel"))) return st;
        }
        if (grad_R) {
            unpack_kernel<<<pack_grid * 2, 256, 0, s>>>(gR, (int32_t)n, ld, w, 1, grad_R, n_sig, c0, nullptr, perm,
                                                        (int32_t)rows);
            if ((st = check_launch("unpack_kernel"))) return st;
        }
    }
    if (g->nnz > 0) {
        edge_grad_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((int32_t)n, g->rowptr, g->colidx, g->sell.sptr,
                                                                     g->sell.iperm, msell, mdiag, (float)two_over_lam,
                                                                     grad_val);
        if ((st = check_launch("edge_grad_kernel"))) return st;
    }
    if (grad_coeffs) {
        SF_CHECK_CUDA(cudaMemcpyAsync(grad_coeffs, ga, sizeof(double) * (p + 1), cudaMemcpyDeviceToHost, s));
        SF_CHECK_CUDA(cudaStreamSynchronize(s));
    }
    return SF_OK;
}
