// The per-order sweep kernel: one sparse product with Lt = (2/lam) L - I
// fused with the three-term Chebyshev recurrence and its epilogue
// (coefficient accumulation, Clenshaw addend, or moment dot products).
//
// Layout: the signal block is processed in column slabs. A slab buffer is
// row-major [N][ld] with ld = LPR * VEC elements, so one row of the slab is
// LPR lanes x 16 bytes; a group of LPR lanes owns a row. The CSR of each tile
// of rows is staged in shared memory by the TMA bulk-copy engine.
#pragma once

#include "sf_internal.cuh"

namespace sf {

// ------------------------------------------------------------ 16-byte vectors
template <typename TS>
struct VT;

template <>
struct VT<float> {
    static constexpr int V = 4;
    __device__ __forceinline__ static void ld_gather(const float *p, float (&x)[4]) {
        float4 v = __ldg(reinterpret_cast<const float4 *>(p));
        x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
    }
    __device__ __forceinline__ static void ld_stream(const float *p, float (&x)[4]) {
        float4 v = __ldcs(reinterpret_cast<const float4 *>(p));
        x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
    }
    __device__ __forceinline__ static void st(float *p, const float (&x)[4]) {
        *reinterpret_cast<float4 *>(p) = make_float4(x[0], x[1], x[2], x[3]);
    }
    __device__ __forceinline__ static void st_cs(float *p, const float (&x)[4]) {
        __stcs(reinterpret_cast<float4 *>(p), make_float4(x[0], x[1], x[2], x[3]));
    }
    __device__ __forceinline__ static void add_raw_mixed(float (&acc)[4], float4 x) { add_raw(acc, x); }
    // value as it is stored (identity for fp32)
    __device__ __forceinline__ static float rt(float x) { return x; }
    __device__ __forceinline__ static float cvt(float x) { return x; }
    using raw_t = float4;
    __device__ __forceinline__ static raw_t ld_raw(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }
    // coherent (L2) load, for blocks written earlier in the same launch
    __device__ __forceinline__ static raw_t ld_raw_cg(const float *p) {
        return __ldcg(reinterpret_cast<const float4 *>(p));
    }
    // the same, read once: evict-first in L2
    __device__ __forceinline__ static raw_t ld_raw_cg_once(const float *p, uint64_t pol) {
        float4 v;
        asm volatile("ld.global.cg.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                     : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                     : "l"(p), "l"(pol));
        return v;
    }
    __device__ __forceinline__ static raw_t zero_raw() { return make_float4(0.f, 0.f, 0.f, 0.f); }
    __device__ __forceinline__ static raw_t ld_raw_stream(const float *p) {
        return __ldcs(reinterpret_cast<const float4 *>(p));
    }
    __device__ __forceinline__ static void to_float(raw_t x, float (&f)[4]) {
        f[0] = x.x; f[1] = x.y; f[2] = x.z; f[3] = x.w;
    }
    __device__ __forceinline__ static void add_raw(float (&acc)[4], raw_t x) {
        acc[0] += x.x;
        acc[1] += x.y;
        acc[2] += x.z;
        acc[3] += x.w;
    }
    // acc += w * x for the 4 values held in a raw register quad
    __device__ __forceinline__ static void fma_raw(float (&acc)[4], float w, raw_t x) {
        acc[0] = fmaf(w, x.x, acc[0]);
        acc[1] = fmaf(w, x.y, acc[1]);
        acc[2] = fmaf(w, x.z, acc[2]);
        acc[3] = fmaf(w, x.w, acc[3]);
    }
};

template <>
struct VT<__nv_bfloat16> {
    static constexpr int V = 8;
    __device__ __forceinline__ static void unpack(uint4 v, float (&x)[8]) {
        const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&v);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float2 f = __bfloat1622float2(h[k]);
            x[2 * k] = f.x;
            x[2 * k + 1] = f.y;
        }
    }
    __device__ __forceinline__ static void ld_gather(const __nv_bfloat16 *p, float (&x)[8]) {
        unpack(__ldg(reinterpret_cast<const uint4 *>(p)), x);
    }
    __device__ __forceinline__ static void ld_stream(const __nv_bfloat16 *p, float (&x)[8]) {
        unpack(__ldcs(reinterpret_cast<const uint4 *>(p)), x);
    }
    __device__ __forceinline__ static uint4 pack(const float (&x)[8]) {
        uint4 v;
        __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(&v);
#pragma unroll
        for (int k = 0; k < 4; ++k) h[k] = __floats2bfloat162_rn(x[2 * k], x[2 * k + 1]);
        return v;
    }
    __device__ __forceinline__ static void st(__nv_bfloat16 *p, const float (&x)[8]) {
        *reinterpret_cast<uint4 *>(p) = pack(x);
    }
    __device__ __forceinline__ static void st_cs(__nv_bfloat16 *p, const float (&x)[8]) {
        __stcs(reinterpret_cast<uint4 *>(p), pack(x));
    }
    __device__ __forceinline__ static float rt(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
    __device__ __forceinline__ static __nv_bfloat16 cvt(float x) { return __float2bfloat16_rn(x); }
    using raw_t = uint4;
    __device__ __forceinline__ static raw_t ld_raw(const __nv_bfloat16 *p) {
        return __ldg(reinterpret_cast<const uint4 *>(p));
    }
    __device__ __forceinline__ static raw_t ld_raw_cg(const __nv_bfloat16 *p) {
        return __ldcg(reinterpret_cast<const uint4 *>(p));
    }
    __device__ __forceinline__ static raw_t ld_raw_cg_once(const __nv_bfloat16 *p, uint64_t pol) {
        uint4 v;
        asm volatile("ld.global.cg.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
                     : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                     : "l"(p), "l"(pol));
        return v;
    }
    __device__ __forceinline__ static raw_t zero_raw() { return make_uint4(0u, 0u, 0u, 0u); }
    __device__ __forceinline__ static raw_t ld_raw_stream(const __nv_bfloat16 *p) {
        return __ldcs(reinterpret_cast<const uint4 *>(p));
    }
    __device__ __forceinline__ static void to_float(raw_t x, float (&f)[8]) {
        const uint32_t h[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            f[2 * k] = __uint_as_float(h[k] << 16);
            f[2 * k + 1] = __uint_as_float(h[k] & 0xffff0000u);
        }
    }
    // a bf16 is the high half of an fp32: widening is a shift or a mask
    __device__ __forceinline__ static void fma_pair(float &a0, float &a1, float w, uint32_t h) {
        a0 = fmaf(w, __uint_as_float(h << 16), a0);
        a1 = fmaf(w, __uint_as_float(h & 0xffff0000u), a1);
    }
    __device__ __forceinline__ static void add_raw(float (&acc)[8], raw_t x) {
        const uint32_t h[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            acc[2 * k] += __uint_as_float(h[k] << 16);
            acc[2 * k + 1] += __uint_as_float(h[k] & 0xffff0000u);
        }
    }
    __device__ __forceinline__ static void fma_raw(float (&acc)[8], float w, raw_t x) {
        fma_pair(acc[0], acc[1], w, x.x);
        fma_pair(acc[2], acc[3], w, x.y);
        fma_pair(acc[4], acc[5], w, x.z);
        fma_pair(acc[6], acc[7], w, x.w);
    }
    // acc += x with the mixed-precision add (FP32 + BF16 operand, one rounding):
    // the same sums as widening first, without the shift and mask
    __device__ __forceinline__ static void add_pair_mixed(float &a0, float &a1, uint32_t h) {
        asm("{\n\t.reg .b16 lo, hi;\n\tmov.b32 {lo, hi}, %2;\n\tadd.rn.f32.bf16 %0, lo, %0;\n\t"
            "add.rn.f32.bf16 %1, hi, %1;\n}"
            : "+f"(a0), "+f"(a1)
            : "r"(h));
    }
    __device__ __forceinline__ static void add_raw_mixed(float (&acc)[8], raw_t x) {
        add_pair_mixed(acc[0], acc[1], x.x);
        add_pair_mixed(acc[2], acc[3], x.y);
        add_pair_mixed(acc[4], acc[5], x.z);
        add_pair_mixed(acc[6], acc[7], x.w);
    }
};

template <>
struct VT<__half> {
    static constexpr int V = 8;
    __device__ __forceinline__ static uint4 pack(const float (&x)[8]) {
        uint4 v;
        __half2 *h = reinterpret_cast<__half2 *>(&v);
#pragma unroll
        for (int k = 0; k < 4; ++k) h[k] = __floats2half2_rn(x[2 * k], x[2 * k + 1]);
        return v;
    }
    __device__ __forceinline__ static void st(__half *p, const float (&x)[8]) {
        *reinterpret_cast<uint4 *>(p) = pack(x);
    }
    __device__ __forceinline__ static void st_cs(__half *p, const float (&x)[8]) {
        __stcs(reinterpret_cast<uint4 *>(p), pack(x));
    }
    __device__ __forceinline__ static float rt(float x) { return __half2float(__float2half_rn(x)); }
    __device__ __forceinline__ static __half cvt(float x) { return __float2half_rn(x); }
    using raw_t = uint4;
    __device__ __forceinline__ static raw_t ld_raw(const __half *p) { return __ldg(reinterpret_cast<const uint4 *>(p)); }
    __device__ __forceinline__ static raw_t ld_raw_cg(const __half *p) {
        return __ldcg(reinterpret_cast<const uint4 *>(p));
    }
    __device__ __forceinline__ static raw_t ld_raw_cg_once(const __half *p, uint64_t pol) {
        uint4 v;
        asm volatile("ld.global.cg.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
                     : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                     : "l"(p), "l"(pol));
        return v;
    }
    __device__ __forceinline__ static raw_t ld_raw_stream(const __half *p) {
        return __ldcs(reinterpret_cast<const uint4 *>(p));
    }
    __device__ __forceinline__ static raw_t zero_raw() { return make_uint4(0u, 0u, 0u, 0u); }
    __device__ __forceinline__ static float2 pair(uint32_t h) {
        return __half22float2(*reinterpret_cast<const __half2 *>(&h));
    }
    __device__ __forceinline__ static void to_float(raw_t x, float (&f)[8]) {
        const uint32_t h[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float2 v = pair(h[k]);
            f[2 * k] = v.x;
            f[2 * k + 1] = v.y;
        }
    }
    __device__ __forceinline__ static void add_raw(float (&acc)[8], raw_t x) {
        const uint32_t h[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float2 v = pair(h[k]);
            acc[2 * k] += v.x;
            acc[2 * k + 1] += v.y;
        }
    }
    __device__ __forceinline__ static void fma_raw(float (&acc)[8], float w, raw_t x) {
        const uint32_t h[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float2 v = pair(h[k]);
            acc[2 * k] = fmaf(w, v.x, acc[2 * k]);
            acc[2 * k + 1] = fmaf(w, v.y, acc[2 * k + 1]);
        }
    }
    __device__ __forceinline__ static void add_pair_mixed(float &a0, float &a1, uint32_t h) {
        asm("{\n\t.reg .b16 lo, hi;\n\tmov.b32 {lo, hi}, %2;\n\tadd.rn.f32.f16 %0, lo, %0;\n\t"
            "add.rn.f32.f16 %1, hi, %1;\n}"
            : "+f"(a0), "+f"(a1)
            : "r"(h));
    }
    __device__ __forceinline__ static void add_raw_mixed(float (&acc)[8], raw_t x) {
        add_pair_mixed(acc[0], acc[1], x.x);
        add_pair_mixed(acc[2], acc[3], x.y);
        add_pair_mixed(acc[4], acc[5], x.z);
        add_pair_mixed(acc[6], acc[7], x.w);
    }
};

// Power-of-two scale that brings the largest magnitude of a block into
// (1/2, 1] (FP16 blocks; 1 when maxbits is null or the block is zero). Being
// a power of two, scaling and unscaling are exact.
__device__ __forceinline__ float block_scale(const uint32_t *maxbits) {
    if (!maxbits) return 1.0f;
    const float mx = __uint_as_float(*maxbits);
    if (!(mx > 0.0f) || isinf(mx)) return 1.0f;
    int e;
    frexpf(mx, &e);  // mx = f * 2^e, f in [1/2, 1)
    return ldexpf(1.0f, -e);
}

// *maxbits = bits of max |R| over the slab's columns [c0, c0 + w)
static __global__ void absmax_kernel(const void *R, int r_dtype, int32_t n, int32_t n_sig, int32_t c0, int32_t w,
                              uint32_t *maxbits) {
    float mx = 0.0f;
    const int64_t total = (int64_t)n * w;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / w;
        const int64_t src = i * n_sig + c0 + (idx - i * w);
        const float x = (r_dtype == SF_BF16) ? __bfloat162float(static_cast<const __nv_bfloat16 *>(R)[src])
                                             : static_cast<const float *>(R)[src];
        mx = fmaxf(mx, fabsf(x));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    // non-negative floats order like their bit patterns
    if ((threadIdx.x & 31) == 0) atomicMax(maxbits, __float_as_uint(mx));
}

// ------------------------------------------------------------ parameters
enum StepMode { MODE_FWD = 0, MODE_MOM = 1, MODE_CLEN = 2 };

// StepParams::flags (uniform per launch)
enum StepFlags {
    STEP_IDX_EVICT_FIRST = 1,  // index copies marked evict-first in L2 (read once per launch)
    STEP_OUT_STREAMING = 2,    // T_j / b_j stores marked streaming (evict-first) instead of write-back
    STEP_MIXED_ADD = 8,        // unit weights, 16-bit blocks: FP32 += 16-bit operand in one instruction
};
constexpr int32_t kStepFlagsDefault = STEP_IDX_EVICT_FIRST | STEP_OUT_STREAMING | STEP_MIXED_ADD;

// Every block (X, Z, Q, out, outf, Y) is row-major in slice-row order
// (sliced-ELL position t = slice * 8 + position, see SellMatrix); rows
// t < n hold graph rows, row `rows` of a gathered block is zero. The per-row
// tables (dtil, wscale, gid) are in the same order.
struct StepParams {
    int32_t n;                 // graph rows: slice rows t >= n are padding and skipped
    const int32_t *sell_ptr;   // sliced-ELL: entry offset of each slice
    const int32_t *sell_idx;   // column indices as slice rows (padding: the zero row)
    const float *sell_val;     // weights (0 for padding), nullptr for unit weights
    const float *dtil;      // per row: 2 s_i / lam - 1
    const float *wscale;    // per row 2 / lam (batches) or nullptr
    float wscale_u;         // uniform 2 / lam
    const int32_t *gid;     // per-row graph id (batches) or nullptr
    int32_t ld;             // slab row stride in elements
    int32_t flags;          // StepFlags
    const void *X;          // T_{j-1} (forward) or b_{j+1} (Clenshaw): gathered
    const void *Z;          // T_{j-2} or b_{j+2}: subtracted (nullptr: none)
    const void *Q;          // Clenshaw addend block (packed R or G)
    void *out;              // T_j or b_j (storage type)
    float *outf;            // Clenshaw final: fp32 output instead of `out`
    float m;                // 2 (general order) or 1 (first order / final Clenshaw step)
    // forward accumulation
    float *Y;               // n_cut accumulators [n_cut][rows][ld] fp32
    int64_t ystride;        // rows * ld
    int32_t n_cut;
    const float *coef;      // [graphs][n_cut][coef_ld]
    int32_t coef_ld;        // p + 1
    int32_t j;              // coefficient index used by this order
    // moments
    double *part;           // [gridDim.x][2]: sum t.t, sum t.x
    double *dots;           // when set: the last block adds the block partials into dots[0..1]
    uint32_t *done;         // blocks finished (zero before the launch; the last block resets it)
    int32_t *status;        // device error word (bit 0: a bounded wait gave up)
};

// ------------------------------------------------------------ async copies
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// 1-D bulk copy global -> shared (TMA engine), completion counted on `bar`.
// dst, src and bytes must be multiples of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
// The same with an L2 cache policy (createpolicy) attached to the reads.
__device__ __forceinline__ void bulk_g2s_hint(void *dst, const void *src, uint32_t bytes, uint64_t *bar,
                                              uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], "
        "%4;" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Programmatic dependent launch: a sweep launched with programmatic stream
// serialization may have its blocks resident while the previous launch in
// the stream is still finishing. Each block signals at its start that the
// next launch may begin (pdl_allow_next) and, before it touches any block,
// accumulator or counter that an earlier launch writes, waits until that
// launch has completed with its memory visible (pdl_wait; it returns at once
// when the launch was not programmatic). Only the CSR (read-only during a
// sweep) is read before the wait.
__device__ __forceinline__ void pdl_allow_next() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Polls are bounded: a copy that never lands makes the kernel record an
// error in *status and return instead of waiting forever.
constexpr uint32_t kWaitPolls = 1u << 22;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    for (uint32_t it = 0; it < kWaitPolls; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// 32-byte FP32 accesses (one 256-bit load or store per lane): with rows in
// slice order, the lanes of a warp cover consecutive 128-byte lines.
__device__ __forceinline__ void ld8_stream(const float *p, float (&x)[8]) {
    asm volatile("ld.global.cs.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=f"(x[0]), "=f"(x[1]), "=f"(x[2]), "=f"(x[3]), "=f"(x[4]), "=f"(x[5]), "=f"(x[6]), "=f"(x[7])
                 : "l"(p));
}
__device__ __forceinline__ void ld8_cg_once(const float *p, float (&x)[8], uint64_t pol) {
    asm volatile("ld.global.cg.L2::cache_hint.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8], %9;"
                 : "=f"(x[0]), "=f"(x[1]), "=f"(x[2]), "=f"(x[3]), "=f"(x[4]), "=f"(x[5]), "=f"(x[6]), "=f"(x[7])
                 : "l"(p), "l"(pol));
}
__device__ __forceinline__ void st8_stream(float *p, const float (&x)[8]) {
    asm volatile("st.global.cs.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "f"(x[0]), "f"(x[1]),
                 "f"(x[2]), "f"(x[3]), "f"(x[4]), "f"(x[5]), "f"(x[6]), "f"(x[7])
                 : "memory");
}

// ------------------------------------------------------------ the sweep
// The sweep reads the graph in a sliced-ELL layout (built from the CSR by
// the library, see sell_build): rows are sorted by length inside windows of
// 32768 rows and grouped into slices of 8 rows padded to a common length (a
// multiple of 4); padding entries point at the zero row appended to every
// gathered block. Each slice is stored row after row, so a row's indices
// are 16-byte aligned and read four at a time. The signal blocks are kept in
// the same (slice-row) order, so the rows a tile streams (its own rows of
// T_{j-1}, T_{j-2}, the output and the accumulators) are consecutive.
//
// A CTA walks tiles of consecutive slices (tile k of the CTA is
// blockIdx.x + k * gridDim.x). A tile's slice offsets and index (and weight)
// range are staged in shared memory by TMA bulk copies into one of NST
// stages. Warps run through the tiles independently: each waits for its
// stage's copy on the stage's mbarrier, and the last warp done with a stage
// (a shared counter) issues the copy of the stage's next tile, so no block
// barrier separates tiles. Tiles whose entries do not fit read the indices
// from global memory. Lane group g (LPR lanes, 16 bytes each) owns tile rows
// g, g + G, ...; the groups of one warp share a slice, so their trip counts
// match.

template <int LPR>
struct TileCfg {
    static constexpr int rows = (LPR == 2) ? 128 : 64;
    static constexpr int slices = rows / kSliceRows;
    static constexpr int sp_ints = slices + 4;  // slices + 1 offsets, rounded up to 16 bytes
    static constexpr int entries = rows * 44;  // 4 blocks of 256 threads fit a 100 KB shared carveout
    static constexpr int stages = 2;
    static constexpr int header = 128;  // mbarriers, per-stage entry base / fits / consumer count / copies issued
    // per stage: slice offsets of the tile and of the stage's next tile (the
    // refill's entry range), indices, weights (weighted graphs only)
    __host__ __device__ static constexpr int buf_bytes(bool weighted) {
        return 2 * sp_ints * 4 + entries * 4 * (weighted ? 2 : 1);
    }
    __host__ __device__ static constexpr int smem_bytes(bool weighted) {
        return header + stages * buf_bytes(weighted);
    }
};

__device__ __forceinline__ int4 lds_int4(const int32_t *p) {
    int4 v;
    asm volatile("ld.shared.v4.s32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"(smem_u32(p)));
    return v;
}
__device__ __forceinline__ float4 lds_float4(const float *p) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(smem_u32(p)));
    return v;
}

template <bool SMEM>
__device__ __forceinline__ int4 ld_idx4(const int32_t *p) {
    if constexpr (SMEM) return lds_int4(p);
    else return __ldg(reinterpret_cast<const int4 *>(p));
}
template <bool SMEM>
__device__ __forceinline__ float4 ld_val4(const float *p) {
    if constexpr (SMEM) return lds_float4(p);
    else return __ldg(reinterpret_cast<const float4 *>(p));
}

// one gathered row chunk: the read-only path, or L2 (COH)
template <typename TS, bool COH>
__device__ __forceinline__ typename VT<TS>::raw_t ld_gathered(const TS *p) {
    if constexpr (COH) return VT<TS>::ld_raw_cg(p);
    else return VT<TS>::ld_raw(p);
}

// acc += sum over the row's ls entries of w_e * X[idx_e] (this lane's 16 bytes).
// COH: the gathered block was written earlier in the same launch, so it is read
// through L2 (the read-only path could hold lines from before the write).
template <typename TS, bool W, bool SMEM, bool MIX, bool COH = false>
__device__ __forceinline__ void gather_row(const TS *__restrict__ Xq, int32_t rstride, const int32_t *ip,
                                           const float *wp, int32_t ls, float (&acc)[VT<TS>::V]) {
    using V = VT<TS>;
    int32_t j = 0;
    for (; j + 8 <= ls; j += 8) {
        const int4 a = ld_idx4<SMEM>(ip + j), b = ld_idx4<SMEM>(ip + j + 4);
        const int32_t k[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
        typename V::raw_t x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = ld_gathered<TS, COH>(Xq + (uint32_t)k[u] * (uint32_t)rstride);
        if constexpr (W) {
            const float4 wa = ld_val4<SMEM>(wp + j), wb = ld_val4<SMEM>(wp + j + 4);
            const float w[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
#pragma unroll
            for (int u = 0; u < 8; ++u) V::fma_raw(acc, w[u], x[u]);
        } else if constexpr (MIX) {
#pragma unroll
            for (int u = 0; u < 8; ++u) V::add_raw_mixed(acc, x[u]);
        } else {
#pragma unroll
            for (int u = 0; u < 8; ++u) V::add_raw(acc, x[u]);
        }
    }
    if (j < ls) {  // ls is a multiple of 4
        const int4 a = ld_idx4<SMEM>(ip + j);
        const int32_t k[4] = {a.x, a.y, a.z, a.w};
        typename V::raw_t x[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) x[u] = ld_gathered<TS, COH>(Xq + (uint32_t)k[u] * (uint32_t)rstride);
        if constexpr (W) {
            const float4 wa = ld_val4<SMEM>(wp + j);
            const float w[4] = {wa.x, wa.y, wa.z, wa.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) V::fma_raw(acc, w[u], x[u]);
        } else if constexpr (MIX) {
#pragma unroll
            for (int u = 0; u < 4; ++u) V::add_raw_mixed(acc, x[u]);
        } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) V::add_raw(acc, x[u]);
        }
    }
}

// The blocks and coefficient index one order works on: from the launch's
// parameters (a launch per order) or from the work item (the persistent batch).
struct OrderView {
    const void *X;  // gathered block
    const void *Z;  // subtracted block (nullptr: none)
    void *out;      // output block
    float *outf;    // Clenshaw final: fp32 output instead of `out`
    float m;        // 2, or 1 for the first order / the final Clenshaw step
    int32_t j;      // coefficient index
};
__device__ __forceinline__ OrderView order_of(const StepParams &P) {
    return OrderView{P.X, P.Z, P.out, P.outf, P.m, P.j};
}

// One row of one order: acc = sum_e w_e X[idx_e] over the row's ls entries,
// then v = m (d_t X_t - (2/lam) acc) - Z_t [+ a_j Q_t], stored; the forward
// mode adds a_cj v to each accumulator, the moment mode sums v.v and v.X_t.
// t is the row's slice-row position, which is also its row in every block.
// COH: every block the launch itself writes is read through L2.
template <typename TS, int MODE, bool W, bool SMEM, bool COH = false>
__device__ __forceinline__ void sweep_row(const StepParams &P, const OrderView &O, int32_t t, int q, const int32_t *ip,
                                          const float *wp, int32_t ls, double &mtt, double &mtx) {
    using V = VT<TS>;
    constexpr int VEC = V::V;
    const TS *__restrict__ X = static_cast<const TS *>(O.X);
    const TS *__restrict__ Z = static_cast<const TS *>(O.Z);
    const TS *__restrict__ Qb = static_cast<const TS *>(P.Q);
    TS *__restrict__ out = static_cast<TS *>(O.out);
    const int32_t ld = P.ld;
    const int64_t ro = (int64_t)t * ld + q * VEC;
    // epilogue operands first (kept packed): their latency overlaps the gathers
    const typename V::raw_t xi_r = ld_gathered<TS, COH>(X + ro);
    typename V::raw_t z_r = V::zero_raw();
    if (Z) {
        // COH: T_{j-2} may still be gathered by tiles of the previous order, so no evict-first hint
        if constexpr (COH) z_r = V::ld_raw_cg(Z + ro);
        else z_r = V::ld_raw_stream(Z + ro);
    }
    typename V::raw_t q_r = V::zero_raw();
    if (MODE == MODE_CLEN) q_r = V::ld_raw_stream(Qb + ro);
    const float d = __ldcs(P.dtil + t);
    const float sc = P.wscale ? __ldcs(P.wscale + t) : P.wscale_u;
    const int g = P.gid ? __ldcs(P.gid + t) : 0;

    float acc[VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v) acc[v] = 0.f;
    if (!W && VEC == 8 && (P.flags & STEP_MIXED_ADD))
        gather_row<TS, W, SMEM, true, COH>(X + q * VEC, ld, ip, wp, ls, acc);
    else gather_row<TS, W, SMEM, false, COH>(X + q * VEC, ld, ip, wp, ls, acc);

    float tv[VEC], xi[VEC];
    {
        float z[VEC];
        V::to_float(xi_r, xi);
        V::to_float(z_r, z);
#pragma unroll
        for (int v = 0; v < VEC; ++v) tv[v] = O.m * fmaf(d, xi[v], -sc * acc[v]) - z[v];
    }
    if (MODE == MODE_CLEN) {
        const float alpha = __ldg(P.coef + (int64_t)g * P.coef_ld + O.j);
        float qv[VEC];
        V::to_float(q_r, qv);
#pragma unroll
        for (int v = 0; v < VEC; ++v) tv[v] = fmaf(alpha, qv[v], tv[v]);
    }
    if (MODE == MODE_CLEN && O.outf) {
        float *o = O.outf + ro;
        if constexpr (VEC == 8) {
            st8_stream(o, tv);
        } else {
            __stcs(reinterpret_cast<float4 *>(o), make_float4(tv[0], tv[1], tv[2], tv[3]));
        }
    } else if (P.flags & STEP_OUT_STREAMING) {
        V::st_cs(out + ro, tv);
    } else {
        V::st(out + ro, tv);
    }
    if (MODE == MODE_FWD) {
        for (int c = 0; c < P.n_cut; ++c) {
            const float a = __ldg(P.coef + ((int64_t)g * P.n_cut + c) * P.coef_ld + O.j);
            float *y = P.Y + c * P.ystride + ro;
            if constexpr (VEC == 8) {
                float yy[8];
                if constexpr (COH) ld8_cg_once(y, yy, l2_policy_evict_first());
                else ld8_stream(y, yy);
#pragma unroll
                for (int v = 0; v < 8; ++v) yy[v] = fmaf(a, tv[v], yy[v]);
                st8_stream(y, yy);
            } else {
                float4 yy = COH ? VT<float>::ld_raw_cg_once(y, l2_policy_evict_first())
                                : __ldcs(reinterpret_cast<const float4 *>(y));
                yy.x = fmaf(a, tv[0], yy.x);
                yy.y = fmaf(a, tv[1], yy.y);
                yy.z = fmaf(a, tv[2], yy.z);
                yy.w = fmaf(a, tv[3], yy.w);
                __stcs(reinterpret_cast<float4 *>(y), yy);
            }
        }
    }
    if (MODE == MODE_MOM) {
        float tt = 0.f, tx = 0.f;
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            const float ts = V::rt(tv[v]);  // the value the next order reads
            tt = fmaf(ts, ts, tt);
            tx = fmaf(ts, xi[v], tx);
        }
        mtt += (double)tt;
        mtx += (double)tx;
    }
}

// Sum over the block of (a, b) in a fixed order (lanes of a warp, then warps);
// the result is valid in thread 0. Every thread of the block calls it.
__device__ __forceinline__ void block_sum2(double &a, double &b, double (*s_red)[2]) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, off);
        b += __shfl_xor_sync(0xffffffffu, b, off);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        s_red[w][0] = a;
        s_red[w][1] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        a = 0.0;
        b = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            a += s_red[k][0];
            b += s_red[k][1];
        }
    }
}

// Moment sums of the block into part[2 * blockIdx.x + {0, 1}]. With P.dots
// set, the block that finishes last adds all block partials, in block order
// (deterministic whichever block is last), into dots[0] and dots[1] and
// resets the counter: no separate reduction launch per order.
__device__ __forceinline__ void block_moments(const StepParams &P, double mtt, double mtx) {
    __shared__ double s_red[32][2];
    __shared__ int s_last;
    block_sum2(mtt, mtx, s_red);
    if (threadIdx.x == 0) {
        P.part[2 * blockIdx.x] = mtt;
        P.part[2 * blockIdx.x + 1] = mtx;
        if (P.dots) {
            __threadfence();  // the partial is visible before the block counts as done
            s_last = (atomicAdd(P.done, 1u) == gridDim.x - 1) ? 1 : 0;
        }
    }
    if (!P.dots) return;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double a = 0.0, b = 0.0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) {
        a += __ldcg(P.part + 2 * k);
        b += __ldcg(P.part + 2 * k + 1);
    }
    __syncthreads();  // s_red is reused
    block_sum2(a, b, s_red);
    if (threadIdx.x == 0) {
        P.dots[0] += a;
        P.dots[1] += b;
        *P.done = 0u;
    }
}

template <typename TS, int LPR, int MODE, bool W>
__global__ void __launch_bounds__(256, 4) cheb_step_kernel(const StepParams P) {
    using C = TileCfg<LPR>;
    constexpr int NST = C::stages;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t *s_bar = reinterpret_cast<uint64_t *>(smem_raw);      // [NST] copy landed
    int32_t *s_meta = reinterpret_cast<int32_t *>(smem_raw + 32);  // [NST][2]: entry base, fits
    int32_t *s_cnt = s_meta + 2 * NST;                              // [NST] warps done with the stage's tile
    int32_t *s_iss = s_cnt + NST;                                   // [NST] copies issued into the stage
    unsigned char *s_buf0 = smem_raw + C::header;
    constexpr int buf_bytes = C::buf_bytes(W);
    static_assert(32 + 4 * NST * 4 <= C::header, "stage header");

    const int tid = threadIdx.x, lane = tid & 31;
    const int q = tid % LPR, grp = tid / LPR;
    const int ngrp = blockDim.x / LPR;
    const int nwarps = blockDim.x >> 5;
    const int n_tiles = (P.n + C::rows - 1) / C::rows;
    double mtt = 0.0, mtx = 0.0;

    // one thread: stage tile `tile` (entries [e0, e1)) into stage b
    auto issue = [&](int tile, int b, int32_t e0, int32_t e1) {
        unsigned char *base = s_buf0 + b * buf_bytes;
        int32_t *sp = reinterpret_cast<int32_t *>(base);
        int32_t *spn = sp + C::sp_ints;
        int32_t *ix = spn + C::sp_ints;
        float *wv = reinterpret_cast<float *>(ix + C::entries);
        const int32_t s0 = tile * C::slices;
        const int next = tile + NST * (int)gridDim.x;  // the stage's tile after this one
        const int32_t cnt = e1 - e0;  // multiple of 32
        const bool fits = cnt <= C::entries;
        const uint32_t bytes = C::sp_ints * 4 * (next < n_tiles ? 2u : 1u) +
                               (fits ? (uint32_t)cnt * 4u * (W ? 2u : 1u) : 0u);
        s_meta[2 * b] = e0;
        s_meta[2 * b + 1] = fits ? 1 : 0;
        s_iss[b] += 1;
        fence_proxy_async();
        mbar_arrive_expect_tx(&s_bar[b], bytes);
        bulk_g2s(sp, P.sell_ptr + s0, C::sp_ints * 4, &s_bar[b]);
        if (next < n_tiles) bulk_g2s(spn, P.sell_ptr + (int64_t)next * C::slices, C::sp_ints * 4, &s_bar[b]);
        if (fits && cnt > 0) {
            if (P.flags & STEP_IDX_EVICT_FIRST) {
                const uint64_t pol = l2_policy_evict_first();
                bulk_g2s_hint(ix, P.sell_idx + e0, cnt * 4, &s_bar[b], pol);
                if (W) bulk_g2s_hint(wv, P.sell_val + e0, cnt * 4, &s_bar[b], pol);
            } else {
                bulk_g2s(ix, P.sell_idx + e0, cnt * 4, &s_bar[b]);
                if (W) bulk_g2s(wv, P.sell_val + e0, cnt * 4, &s_bar[b]);
            }
        }
    };

    pdl_allow_next();
    if (tid == 0) {
        for (int b = 0; b < NST; ++b) {
            mbar_init(&s_bar[b], 1);
            s_cnt[b] = 0;
            s_iss[b] = 0;
        }
        fence_mbar_init();
        for (int b = 0; b < NST; ++b) {
            const int tile = blockIdx.x + b * gridDim.x;
            if (tile < n_tiles) issue(tile, b, P.sell_ptr[tile * C::slices], P.sell_ptr[(tile + 1) * C::slices]);
        }
    }
    __syncthreads();
    pdl_wait();  // the first tiles' CSR copies overlap the previous launch's end
    for (int k = 0;; ++k) {
        const int tile = blockIdx.x + k * gridDim.x;
        if (tile >= n_tiles) break;
        const int b = k % NST;
        const uint32_t par = (uint32_t)(k / NST) & 1u;
        if (!mbar_wait_bounded(&s_bar[b], par)) {
            if (lane == 0) atomicOr(P.status, 1);
            break;  // the other warps give up on their own waits; copies in flight are awaited below
        }
        const int32_t *s_sp = reinterpret_cast<const int32_t *>(s_buf0 + b * buf_bytes);
        const int32_t *s_ix = s_sp + 2 * C::sp_ints;
        const float *s_wv = reinterpret_cast<const float *>(s_ix + C::entries);
        const int32_t e0 = s_meta[2 * b];
        const bool fits = s_meta[2 * b + 1] != 0;

        for (int tr = grp; tr < C::rows; tr += ngrp) {
            const int32_t t = tile * C::rows + tr;
            if (t >= P.n) continue;  // padding rows of the last tile
            const int sl = tr / kSliceRows, pos = tr % kSliceRows;
            const int32_t so = s_sp[sl], ls = (s_sp[sl + 1] - so) / kSliceRows;
            const int32_t eo = so - e0 + pos * ls;  // offset of the row's first entry in the tile
            if (fits) sweep_row<TS, MODE, W, true>(P, order_of(P), t, q, s_ix + eo, s_wv + eo, ls, mtt, mtx);
            else sweep_row<TS, MODE, W, false>(P, order_of(P), t, q, P.sell_idx + e0 + eo,
                                               W ? P.sell_val + e0 + eo : nullptr, ls, mtt, mtx);
        }
        __syncwarp();
        if (lane == 0) {
            __threadfence_block();  // this warp's reads of the stage come before its release
            if (atomicAdd(&s_cnt[b], 1) == nwarps - 1) {
                // the last warp done with the stage refills it with the stage's next tile,
                // whose entry range came with this tile's copy
                __threadfence_block();  // every warp's reads of the stage come before the refill
                s_cnt[b] = 0;
                const int next = tile + NST * (int)gridDim.x;
                if (next < n_tiles) {
                    const int32_t *spn = s_sp + C::sp_ints;
                    issue(next, b, spn[0], spn[C::slices]);
                }
            }
        }
    }
    __syncthreads();
    if (tid == 0) {
        // after a wait gave up, copies may still be in flight: wait (bounded) for the last one of each stage
        for (int b = 0; b < NST; ++b)
            if (s_iss[b] > 0) mbar_wait_bounded(&s_bar[b], (uint32_t)(s_iss[b] - 1) & 1u);
    }
    if (MODE == MODE_MOM) block_moments(P, mtt, mtx);
}

// Direct variant: no staging and no block barriers. Warp c of the grid walks
// chunks of 32 / LPR consecutive slice rows (chunk c, c + W, ... for W warps
// in the grid); each lane group reads its row's slice offsets and indices
// straight from global memory (16-byte vector loads, broadcast within the
// group). With no shared memory the whole L1 holds gathers in flight.
template <typename TS, int LPR, int MODE, bool W>
__global__ void __launch_bounds__(256, 4) cheb_step_direct_kernel(const StepParams P) {
    pdl_allow_next();
    pdl_wait();
    constexpr int RPW = 32 / LPR;
    const int lane = threadIdx.x & 31, q = lane % LPR, g = lane / LPR;
    const int64_t n_chunks = ((int64_t)P.n + RPW - 1) / RPW;
    const int wpb = blockDim.x >> 5;
    const int64_t warps = (int64_t)gridDim.x * wpb;
    double mtt = 0.0, mtx = 0.0;
    for (int64_t c = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); c < n_chunks; c += warps) {
        const int64_t t = c * RPW + g;
        if (t >= P.n) continue;
        const int32_t sl = (int32_t)(t / kSliceRows), pos = (int32_t)(t % kSliceRows);
        const int32_t so = __ldg(P.sell_ptr + sl);
        const int32_t ls = (__ldg(P.sell_ptr + sl + 1) - so) / kSliceRows;
        const int64_t eo = (int64_t)so + (int64_t)pos * ls;
        sweep_row<TS, MODE, W, false>(P, order_of(P), (int32_t)t, q, P.sell_idx + eo,
                                      W ? P.sell_val + eo : nullptr, ls, mtt, mtx);
    }
    if (MODE == MODE_MOM) block_moments(P, mtt, mtx);
}

// ------------------------------------------------------------ persistent batch
// One launch filters a batch of graphs through all p orders. Work item
// i = s * n_chunks + c is order step s (forward: order s + 1; Clenshaw:
// index j = p - 1 - s) of chunk c, `chunk` consecutive tiles. Blocks claim
// items from a global counter in increasing order, and an item may start once
// every graph its chunk covers has completed step s - 1 on all of that
// graph's chunks (per-graph arrival counters). Every item an item waits for
// has a smaller index, so it was claimed before by a block that is running:
// the launch cannot deadlock, whatever the grid. A small graph therefore moves
// to its next order as soon as its own chunks are done, without waiting for
// the rest of the batch. Each wait is bounded; one that gives up sets the
// status word and an abort flag that makes every other wait give up at once.
// The thread that claims an item polls its counters once; when they are
// already complete the item's first tile arrives marked ready and the warps
// skip their own wait.
constexpr int kBatchChunk = 8;  // most tiles per work item

struct BatchSched {
    int32_t n_tiles;
    int32_t chunk;                // tiles per work item, 1..kBatchChunk
    int32_t n_chunks;             // ceil(n_tiles / chunk)
    int32_t p;                    // orders: the launch runs p steps
    const int32_t *chunk_glo;     // [n_chunks] lowest graph id among the chunk's rows
    const int32_t *chunk_ghi;     // [n_chunks] highest graph id among the chunk's rows
    const uint32_t *graph_chunks; // [n_graphs] chunks whose graph range covers the graph
    uint32_t *done;               // [n_graphs] completed items covering the graph (zero at launch)
    uint32_t *queue;              // next item to claim (zero at launch)
    int32_t *abort;               // nonzero once any wait gave up (zero at launch)
    void *buf[3];                 // the three rotating blocks (rows + 1 rows each)
};

// buf[k % 3] by selects (a dynamic index into the parameter array would go through local memory)
__device__ __forceinline__ void *sched_buf(const BatchSched &S, int k) {
    const int r = k % 3;
    return r == 0 ? S.buf[0] : (r == 1 ? S.buf[1] : S.buf[2]);
}

template <int MODE>
__device__ __forceinline__ OrderView order_at(const StepParams &P, const BatchSched &S, int s) {
    OrderView O;
    if (MODE == MODE_FWD) {
        const int j = s + 1;
        O.X = sched_buf(S, j - 1);
        O.Z = (j >= 2) ? sched_buf(S, j - 2) : nullptr;
        O.out = sched_buf(S, j);
        O.outf = nullptr;
        O.m = (j == 1) ? 1.0f : 2.0f;
        O.j = j;
    } else {
        const int j = S.p - 1 - s;
        O.X = sched_buf(S, j + 1);
        O.Z = (j + 2 <= S.p) ? sched_buf(S, j + 2) : nullptr;
        O.out = (j == 0) ? nullptr : sched_buf(S, j);
        O.outf = (j == 0) ? P.outf : nullptr;
        O.m = (j == 0) ? 1.0f : 2.0f;
        O.j = j;
    }
    return O;
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int32_t ld_volatile_i32(const int32_t *p) {
    return *reinterpret_cast<const volatile int32_t *>(p);
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

constexpr uint32_t kDepPolls = 1u << 20;  // with a 128 ns sleep between polls: about a second

// One poll: has every graph of chunk c completed step s - 1?
__device__ __forceinline__ bool graph_deps_done(const BatchSched &S, int s, int c) {
    if (s == 0) return true;
    const int g0 = __ldg(S.chunk_glo + c), g1 = __ldg(S.chunk_ghi + c);
    for (int g = g0; g <= g1; ++g)
        if (ld_acquire_u32(S.done + g) < (uint32_t)s * __ldg(S.graph_chunks + g)) return false;
    return true;
}

// Waits (at most `polls` polls per graph) until every graph of chunk c has
// completed step s - 1.
__device__ __forceinline__ bool wait_graph_deps(const BatchSched &S, int s, int c, uint32_t polls = kDepPolls) {
    if (s == 0) return true;
    const int g0 = __ldg(S.chunk_glo + c), g1 = __ldg(S.chunk_ghi + c);
    for (int g = g0; g <= g1; ++g) {
        const uint32_t need = (uint32_t)s * __ldg(S.graph_chunks + g);
        uint32_t it = 0;
        while (ld_acquire_u32(S.done + g) < need) {
            if (++it >= polls || ld_volatile_i32(S.abort)) return false;
            __nanosleep(128);
        }
    }
    return true;
}

// Stage wait that also gives up as soon as another wait of the launch did.
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t *bar, uint32_t parity, const int32_t *abort) {
    for (uint32_t it = 0; it < kWaitPolls; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255u) == 255u && ld_volatile_i32(abort)) return false;
    }
    return false;
}

// The block's tiles form a sequence (the tiles of its items in claim order);
// the two stages hold consecutive positions of it. s_pos[b] = (item, tile of
// the item, ready) staged in stage b (item -1: the queue is exhausted); s_cur
// = the next position to stage. The next item is claimed, and its counters
// polled once, right after the copy of the current item's last tile is
// issued (s_next = item, ready), so neither round trip delays a stage.
// ready: the item's dependencies were complete when polled; the polling
// thread's acquire reaches the warps through the stage counters' CTA fences
// and the stage mbarrier's release/acquire.
template <typename TS, int LPR, int MODE, bool W>
__global__ void __launch_bounds__(256, 4) cheb_batch_kernel(const StepParams P, const BatchSched S) {
    using C = TileCfg<LPR>;
    constexpr int NST = C::stages;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t *s_bar = reinterpret_cast<uint64_t *>(smem_raw);      // [NST] copy landed
    int32_t *s_meta = reinterpret_cast<int32_t *>(smem_raw + 32);  // [NST][2]: entry base, fits
    int32_t *s_cnt = s_meta + 2 * NST;                              // [NST] warps done with the stage's tile
    int32_t *s_iss = s_cnt + NST;                                   // [NST] phases started on the stage
    int32_t *s_pos = s_iss + NST;                                   // [NST][3]: item, tile of the item, ready
    int32_t *s_cur = s_pos + 3 * NST;                               // [2]: the next position to stage
    int32_t *s_next = s_cur + 2;                                    // [2]: the claimed next item, ready
    unsigned char *s_buf0 = smem_raw + C::header;
    constexpr int buf_bytes = C::buf_bytes(W);
    static_assert(32 + 8 * NST * 4 + 16 <= C::header, "stage header");

    const int tid = threadIdx.x, lane = tid & 31;
    const int q = tid % LPR, grp = tid / LPR;
    const int ngrp = blockDim.x / LPR;
    const int nwarps = blockDim.x >> 5;
    const int total = S.p * S.n_chunks;
    double mtt = 0.0, mtx = 0.0;  // unused (no moment mode for batches)

    // tiles of chunk c
    auto chunk_tiles = [&](int c) {
        const int t0 = c * S.chunk;
        return (S.n_tiles - t0) < S.chunk ? (S.n_tiles - t0) : S.chunk;
    };
    // one thread: claim the next item and poll its dependencies once
    auto claim_next = [&]() {
        const int it = (int)atomicAdd(S.queue, 1u);
        const int item = (it < total) ? it : -1;
        s_next[0] = item;
        s_next[1] = (item >= 0 && graph_deps_done(S, item / S.n_chunks, item % S.n_chunks)) ? 1 : 0;
    };
    // one thread: stage the sequence's next tile into stage b (or mark the
    // stage exhausted), moving to the claimed item when the current one is
    // used up; after the copy of an item's last tile, claim the next item
    auto stage_next = [&](int b) {
        int item = s_cur[0], k = s_cur[1];
        int ready = 1;
        if (item < 0 || k >= chunk_tiles(item % S.n_chunks)) {
            item = s_next[0];
            ready = s_next[1];
            k = 0;
        }
        s_cur[0] = item;
        s_cur[1] = k + 1;
        s_pos[3 * b] = item;
        s_pos[3 * b + 1] = k;
        s_pos[3 * b + 2] = ready;
        s_iss[b] += 1;
        if (item < 0) {
            mbar_arrive(&s_bar[b]);
            return;
        }
        const int tile = (item % S.n_chunks) * S.chunk + k;
        unsigned char *base = s_buf0 + b * buf_bytes;
        int32_t *sp = reinterpret_cast<int32_t *>(base);
        int32_t *ix = sp + 2 * C::sp_ints;
        float *wv = reinterpret_cast<float *>(ix + C::entries);
        const int32_t s0 = tile * C::slices;
        const int32_t e0 = __ldg(P.sell_ptr + s0), e1 = __ldg(P.sell_ptr + s0 + C::slices);
        const int32_t cnt = e1 - e0;
        const bool fits = cnt <= C::entries;
        const uint32_t bytes = C::sp_ints * 4 + (fits ? (uint32_t)cnt * 4u * (W ? 2u : 1u) : 0u);
        s_meta[2 * b] = e0;
        s_meta[2 * b + 1] = fits ? 1 : 0;
        fence_proxy_async();
        mbar_arrive_expect_tx(&s_bar[b], bytes);
        bulk_g2s(sp, P.sell_ptr + s0, C::sp_ints * 4, &s_bar[b]);
        if (fits && cnt > 0) {
            if (P.flags & STEP_IDX_EVICT_FIRST) {
                const uint64_t pol = l2_policy_evict_first();
                bulk_g2s_hint(ix, P.sell_idx + e0, cnt * 4, &s_bar[b], pol);
                if (W) bulk_g2s_hint(wv, P.sell_val + e0, cnt * 4, &s_bar[b], pol);
            } else {
                bulk_g2s(ix, P.sell_idx + e0, cnt * 4, &s_bar[b]);
                if (W) bulk_g2s(wv, P.sell_val + e0, cnt * 4, &s_bar[b]);
            }
        }
        if (k + 1 >= chunk_tiles(item % S.n_chunks)) claim_next();
    };

    if (tid == 0) {
        for (int b = 0; b < NST; ++b) {
            mbar_init(&s_bar[b], 1);
            s_cnt[b] = 0;
            s_iss[b] = 0;
        }
        s_cur[0] = -1;
        s_cur[1] = 0;
        fence_mbar_init();
        claim_next();
        for (int b = 0; b < NST; ++b) stage_next(b);
    }
    __syncthreads();
    for (int k = 0;; ++k) {
        const int b = k % NST;
        const uint32_t par = (uint32_t)(k / NST) & 1u;
        if (!mbar_wait_or_abort(&s_bar[b], par, S.abort)) {
            if (lane == 0) {
                atomicOr(P.status, 1);
                atomicExch(S.abort, 1);
            }
            break;
        }
        const int item = s_pos[3 * b], kt = s_pos[3 * b + 1];
        if (item < 0) break;  // the queue is exhausted
        const int s = item / S.n_chunks, c = item % S.n_chunks;
        const int tile = c * S.chunk + kt;
        if (kt == 0 && !s_pos[3 * b + 2]) {  // the item's first tile: its graphs must have finished the previous step
            bool ok = true;
            if (lane == 0) {
                ok = wait_graph_deps(S, s, c);
                if (!ok) {
                    atomicOr(P.status, 2);
                    atomicExch(S.abort, 1);
                }
            }
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            __syncwarp();  // lane 0's acquire of the counters is ordered before every lane's reads below
            if (!ok) break;
        }
        const OrderView O = order_at<MODE>(P, S, s);
        const int32_t *s_sp = reinterpret_cast<const int32_t *>(s_buf0 + b * buf_bytes);
        const int32_t *s_ix = s_sp + 2 * C::sp_ints;
        const float *s_wv = reinterpret_cast<const float *>(s_ix + C::entries);
        const int32_t e0 = s_meta[2 * b];
        const bool fits = s_meta[2 * b + 1] != 0;
        for (int tr = grp; tr < C::rows; tr += ngrp) {
            const int32_t t = tile * C::rows + tr;
            if (t >= P.n) continue;
            const int sl = tr / kSliceRows, pos = tr % kSliceRows;
            const int32_t so = s_sp[sl], ls = (s_sp[sl + 1] - so) / kSliceRows;
            const int32_t eo = so - e0 + pos * ls;
            if (fits) sweep_row<TS, MODE, W, true, true>(P, O, t, q, s_ix + eo, s_wv + eo, ls, mtt, mtx);
            else sweep_row<TS, MODE, W, false, true>(P, O, t, q, P.sell_idx + e0 + eo,
                                                     W ? P.sell_val + e0 + eo : nullptr, ls, mtt, mtx);
        }
        __syncwarp();
        if (lane == 0) {
            __threadfence_block();  // this warp's rows come before its release of the stage
            if (atomicAdd(&s_cnt[b], 1) == nwarps - 1) {
                __threadfence_block();
                s_cnt[b] = 0;
                if (kt == chunk_tiles(c) - 1) {
                    // the item is complete: release every warp's rows to the GPU, then count the
                    // item for every graph its chunk covers
                    fence_acq_rel_gpu();
                    const int g0 = __ldg(S.chunk_glo + c), g1 = __ldg(S.chunk_ghi + c);
                    for (int g = g0; g <= g1; ++g) atomicAdd(S.done + g, 1u);
                }
                stage_next(b);
            }
        }
    }
    __syncthreads();
    if (tid == 0) {
        // copies may still be in flight after a wait gave up: wait (bounded) for the last one of each stage
        for (int b = 0; b < NST; ++b)
            if (s_iss[b] > 0) mbar_wait_bounded(&s_bar[b], (uint32_t)(s_iss[b] - 1) & 1u);
    }
}

// ------------------------------------------------------------ pack / unpack
// Blocks hold rows in slice-row order: block row t is graph row perm[t]
// (perm[t] < 0 and t >= rows: zero rows). pack_kernel fills rows
// [0, rows] of T0 with the R slab converted to the storage type (zero padded
// to ld columns). Optionally: Y_c = a_c0 * T0 (forward, rows [0, rows)),
// b_p = a_p * T0 (Clenshaw start, written to `bstart`), and per-block
// partial sum of T0.T0 (moments). gid is indexed by graph row.
//
// Elements are taken in block order, kPackUnroll per lane per pass (their
// loads issued together, so that a pass keeps that many reads in flight); a
// warp's 32 x kPackUnroll elements are summed in FP32, then in FP64 across
// passes and warps in a fixed order. ld is a power of two.
constexpr int kPackUnroll = 8;
constexpr int kPackBlocksPerSm = 8;  // pack/unpack grids: kPackBlocksPerSm x SMs blocks of 256 threads

template <typename TS>
__global__ void __launch_bounds__(256) pack_kernel(const void *R, int r_dtype, int32_t n, int32_t n_sig, int32_t c0,
                                                   int32_t w, int32_t ld, TS *T0, float *Y, int64_t ystride,
                                                   int32_t n_cut, const float *coef, int32_t coef_ld, int32_t jcoef,
                                                   const int32_t *gid, TS *bstart, double *part,
                                                   const uint32_t *maxbits, const int32_t *perm, int32_t rows) {
    __shared__ double red[8];
    const int lane = threadIdx.x & 31;
    const int lg = __ffs(ld) - 1;
    const int64_t total = (int64_t)(rows + 1) * ld;
    const float scale = block_scale(maxbits);
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    constexpr int64_t kSpan = 32 * kPackUnroll;
    double acc = 0.0;
    for (int64_t base = warp0 * kSpan; base < total; base += nwarps * kSpan) {
        float x[kPackUnroll];
        int32_t iv[kPackUnroll];
#pragma unroll
        for (int u = 0; u < kPackUnroll; ++u) {
            const int64_t idx = base + u * 32 + lane;
            const int64_t t = idx >> lg;
            const int32_t c = (int32_t)(idx & (ld - 1));
            const int32_t i = (idx < total && t < rows) ? __ldg(perm + t) : -1;
            iv[u] = i;
            x[u] = 0.f;
            if (i >= 0 && c < w) {
                const int64_t src = (int64_t)i * n_sig + c0 + c;
                x[u] = (r_dtype == SF_BF16) ? __bfloat162float(static_cast<const __nv_bfloat16 *>(R)[src])
                                            : __ldg(static_cast<const float *>(R) + src);
            }
        }
        float ss = 0.f;
#pragma unroll
        for (int u = 0; u < kPackUnroll; ++u) {
            const int64_t idx = base + u * 32 + lane;
            if (idx >= total) continue;
            const float xs = x[u] * scale;
            T0[idx] = VT<TS>::cvt(xs);
            const float xr = VT<TS>::rt(xs);
            ss = fmaf(xr, xr, ss);
            if ((idx >> lg) == rows) continue;  // the zero row of the gathered block
            const int32_t i = iv[u];
            const int g = (gid && i >= 0) ? __ldg(gid + i) : 0;
            if (Y) {
                for (int k = 0; k < n_cut; ++k) {
                    const float a = __ldg(coef + ((int64_t)g * n_cut + k) * coef_ld + jcoef);
                    Y[k * ystride + idx] = a * xr;
                }
            }
            if (bstart) {
                const float a = __ldg(coef + (int64_t)g * coef_ld + jcoef);
                bstart[idx] = VT<TS>::cvt(a * xr);
            }
        }
        if (part) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, off);
            acc += (double)ss;  // the same in every lane
        }
    }
    if (part) {
        if (lane == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double sum = 0.0;
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k) sum += red[k];
            part[blockIdx.x] = sum;
        }
    }
}

// Y_out[c][perm[t]][c0 + col] = Yslab[c][t][col] for col < w and graph rows t
// (kPackUnroll elements per lane per pass, in block order; ld a power of two).
static __global__ void __launch_bounds__(256) unpack_kernel(const float *Yslab, int32_t n, int32_t ld, int32_t w,
                                                            int32_t n_cut, float *Y, int32_t n_sig, int32_t c0,
                                                            const uint32_t *maxbits, const int32_t *perm,
                                                            int32_t rows) {
    const int lane = threadIdx.x & 31;
    const int lg = __ffs(ld) - 1;
    const int64_t per_cut = (int64_t)rows * ld;
    const float inv = 1.0f / block_scale(maxbits);  // exact: a power of two
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    constexpr int64_t kSpan = 32 * kPackUnroll;
    for (int32_t cc = 0; cc < n_cut; ++cc) {
        const float *src = Yslab + cc * per_cut;
        float *dst = Y + (int64_t)cc * n * n_sig + c0;
        for (int64_t base = warp0 * kSpan; base < per_cut; base += nwarps * kSpan) {
            float v[kPackUnroll];
            int32_t iv[kPackUnroll];
#pragma unroll
            for (int u = 0; u < kPackUnroll; ++u) {
                const int64_t idx = base + u * 32 + lane;
                const int32_t c = (int32_t)(idx & (ld - 1));
                iv[u] = (idx < per_cut && c < w) ? __ldg(perm + (idx >> lg)) : -1;
                v[u] = iv[u] >= 0 ? __ldcs(src + idx) : 0.f;
            }
#pragma unroll
            for (int u = 0; u < kPackUnroll; ++u) {
                const int64_t idx = base + u * 32 + lane;
                if (iv[u] >= 0) dst[(int64_t)iv[u] * n_sig + (idx & (ld - 1))] = v[u] * inv;
            }
        }
    }
}

// Per slice row t (graph row i = perm[t]): d~_t = 2 s_i / lam - 1 (uniform lam)
// or with the graph's own lam (batches), 2 / lam per row for batches, and the
// graph id per row; padding rows get zeros.
static __global__ void dtil_kernel(const double *s, int32_t rows, double two_over_lam, const int32_t *gid,
                                   const double *two_over_lam_g, float *dtil, float *wscale, const int32_t *perm,
                                   int32_t *gid_t) {
    int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= rows) return;
    const int32_t i = perm[t];
    if (i < 0) {
        dtil[t] = 0.0f;
        if (wscale) wscale[t] = 0.0f;
        if (gid_t) gid_t[t] = 0;
        return;
    }
    const int g = gid ? gid[i] : 0;
    double tl = gid ? two_over_lam_g[g] : two_over_lam;
    dtil[t] = (float)(tl * s[i] - 1.0);
    if (wscale) wscale[t] = (float)tl;
    if (gid_t) gid_t[t] = g;
}

// Sum the [count][2] partials in a fixed order and add into out[0..1].
static __global__ void pair_sum_kernel(const double *part, int32_t count, int32_t stride, double *out) {
    __shared__ double a[256], b[256];
    double x = 0.0, y = 0.0;
    for (int k = threadIdx.x; k < count; k += blockDim.x) {
        x += part[(int64_t)k * stride];
        if (stride == 2) y += part[(int64_t)k * 2 + 1];
    }
    a[threadIdx.x] = x;
    b[threadIdx.x] = y;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            a[threadIdx.x] += a[threadIdx.x + s];
            b[threadIdx.x] += b[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] += a[0];
        if (stride == 2) out[1] += b[0];
    }
}

// ------------------------------------------------------------ host side
struct SweepShape {
    int storage;      // SF_F32 / SF_BF16 / SF_F16
    int lpr;          // lanes per row-chunk
    int ld;           // slab columns (= lpr * vec)
    int block;        // threads per block
    int grid;         // blocks
    int smem;         // dynamic shared memory per block
    bool weighted;    // kernel reads weights
    bool direct = false;  // cheb_step_direct_kernel instead of the staged tiles
    size_t l2_window_bytes = 0;  // persisting-L2 window over the gathered block (0: none)
    float l2_hit_ratio = 0.f;
};

// Picks the slab width (columns) for n rows and n_sig signals.
int auto_slab_cols(int64_t n, int n_sig, int storage, int64_t l2_budget_bytes);
constexpr int64_t kAutoSlabBudget = 64ll << 20;  // gathered block per slab: about half of L2
sf_status make_shape(int storage, int slab_cols, int block_warps, int blocks_per_sm, int mode, bool weighted,
                     SweepShape *sh, int carveout_pct = 0, int sweep_kernel = 0);
using StepFn = void (*)(const StepParams);
// cheb_step_direct_kernel instances (defined in their own translation unit).
StepFn direct_step_fn(int storage, int lpr, int mode, bool weighted);
// Device error word written by the sweep kernels (bounded waits).
int32_t *device_status();
sf_status launch_step(const SweepShape &sh, int mode, const StepParams &P, cudaStream_t s, double bytes);
// StepParams::flags for a call's options (sf_opts.sweep_hints).
int32_t step_flags(const sf_opts &o);
// Finiteness and growth checks of a moment sweep's dot products (SF_ERR_NUMERIC).
sf_status check_moment_dots(const double *dots, double e_last, int p, double lam_max);

// The persistent batch sweep (sf_batch.cu): all p orders of one column slab
// of a batch in one launch. gid_t holds the graph id of each slice row; P is
// set up as for the per-order launches (P.outf: the Clenshaw output block).
sf_status make_batch_shape(int storage, int slab_cols, int block_warps, int blocks_per_sm, int mode, bool weighted,
                           int carveout_pct, SweepShape *sh);
sf_status launch_batch_persistent(const SweepShape &sh, int mode, StepParams P, int32_t n_graphs, int32_t p,
                                  const int32_t *gid_t, void *const buf[3], cudaStream_t s, double bytes);

}  // namespace sf
