// k-means on the feature rows (§4.1 step 6: k-means with the Euclidean
// distance between rows f~_i), Lloyd's iterations from given centroids.
//
// Assignment. The label of row i is argmin_c d(f_i, c_c), ties to the lowest
// c, where d is the FP32 sum of fused multiply-adds (f_j - c_j)^2 in index
// order: a floating-point decision, so it is stated in one precision and
// order. Two ways to take it:
//  * CUDA cores: exactly that sum, in km_assign_blocked_kernel (32 rows x 128
//    centroids per block, register tiles; k <= 128, d <= 256) or else
//    km_assign_kernel (a warp per row, a lane per centroid);
//  * tensor cores (kmeans_tc_kernel): G = F C^T for a 128-row tile on tcgen05
//    (TF32 operands staged by TMA in 128-byte swizzled shared memory, FP32
//    accumulators in TMEM), e_c = |c_c|^2 - 2 G_ic; the row takes the tensor
//    argmin when its two best candidates are further apart than twice the
//    bound on |e_c + |f_i|^2 - d(f_i, c_c)|, and is otherwise queued with a
//    superset of the centroids within that margin of its best (no other
//    centroid can win in FP32), which km_assign_cands_kernel then decides
//    exactly. Both give the same labels.
// Bound, one product per pair (F and C as given, read as TF32): TF32 keeps
// 10 mantissa bits (truncation error < 2^-10 per operand), so
// |G_ic - f_i.c_c| <= (2^-9 + 2^-16) |f_i| |c_c| with FP32 accumulation of
// 128 products; |c|^2 and the FP32 sum d carry <= 2^-16 (|f| + |c|)^2. With
// the factor 2 on G and a safety margin: E_i = 2^-7 |f_i| c_max +
// 2^-16 (|f_i| + c_max)^2, and a row is decided by the tensor cores when the
// gap between its two best e exceeds 2 E_i.
// Split operands (the default): x = hi + lo + r with hi, lo TF32 (round to
// nearest) and |r| <= 2^-22 |x|; G = hi.hi + hi.lo + lo.hi drops terms of at
// most 3.01 2^-22 |f||c| in all, and the FP32 accumulation of 3 d <= 384
// exact TF32 products (1 ulp per addition) adds <= 2^-14.4 |f||c|: with the
// factor 2 and a safety margin the first term of E_i becomes 2^-12 |f_i| c_max.
//
// Update. c_c = (sum of its rows / count) rounded to FP32, an empty cluster
// keeping its centroid. The sums are exact integer sums of the values
// rounded down to multiples of 2^-sh, with 2^sh as large as keeps
// n max|F_ij| 2^sh below 2^62 (an absolute error below n 2^-sh <=
// 2^-60 n^2 max|F_ij| per sum, under the bound of about 2^-53 n^2 max|F_ij|
// of an FP64 sum in row order); integer addition is associative, so blocks
// and atomics may add in any order and the centroids are deterministic.
#include <cuda.h>

#include <algorithm>
#include <math.h>

#include "sf_step.cuh"

namespace sf {

constexpr int kTcRows = 128;  // rows of F per tensor-core tile (MMA M)

// ------------------------------------------------------------ small kernels
// |f_i| (FP32, rounded up by 2^-20 relative), a warp per four rows (their
// loads in flight together); fmax_bits: the largest |F_ij| (float bits,
// atomicMax of non-negative floats as ints)
__global__ void km_row_norm_kernel(const float *F, int32_t n, int32_t d, float *fn, int32_t *bad,
                                   int32_t *fmax_bits) {
    const int lane = threadIdx.x & 31;
    float mx = 0.f;
    for (int64_t i0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 4; i0 < n;
         i0 += (((int64_t)gridDim.x * blockDim.x) >> 5) * 4) {
        float s[4] = {0.f, 0.f, 0.f, 0.f};
        for (int j = lane; j < d; j += 32) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float x = (i0 + u < n) ? F[(i0 + u) * d + j] : 0.f;
                s[u] = fmaf(x, x, s[u]);
                mx = fmaxf(mx, fabsf(x));
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) s[u] += __shfl_xor_sync(0xffffffffu, s[u], off);
        }
        if (lane < 4 && i0 + lane < n) {
            const float v = lane == 0 ? s[0] : lane == 1 ? s[1] : lane == 2 ? s[2] : s[3];
            fn[i0 + lane] = sqrtf(v) * (1.0f + 1.0f / 1048576.0f);
            if (!isfinite(v)) *bad = 1;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if (lane == 0 && mx > 0.f) atomicMax(fmax_bits, __float_as_int(mx));
}

// cn2[c] = |c_c|^2 (FP32 fused multiply-adds in index order); cmax = max |c| rounded up. One block.
__global__ void km_centroid_norm_kernel(const float *C, int32_t k, int32_t d, float *cn2, float *cmax,
                                        int32_t *bad) {
    __shared__ float s_max[32];
    float mx = 0.f;
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        float s = 0.f;
        for (int j = 0; j < d; ++j) s = fmaf(C[(int64_t)c * d + j], C[(int64_t)c * d + j], s);
        cn2[c] = s;
        mx = fmaxf(mx, s);
        if (!isfinite(s)) *bad = 1;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, s_max[w]);
        *cmax = sqrtf(m) * (1.0f + 1.0f / 1048576.0f);
    }
}

// The exact decision for one row: lane l scores centroids l, l + 32, ...
// (each an FP32 fused-multiply-add chain in index order), then the warp keeps
// the smallest score, ties to the lowest centroid. sC: centroids with row
// stride ldc (a shared-memory copy, or C itself).
__device__ __forceinline__ int32_t km_decide_row(const float *__restrict__ f, const float *sC, int32_t ldc, int32_t k,
                                                 int32_t d, float *best_d) {
    const int lane = threadIdx.x & 31;
    float bd = INFINITY;
    int32_t bc = 0x7fffffff;
    for (int c = lane; c < k; c += 32) {
        const float *cc = sC + (int64_t)c * ldc;
        float acc = 0.f;
        for (int j = 0; j < d; ++j) {
            const float t = __fsub_rn(__ldg(f + j), cc[j]);
            acc = __fmaf_rn(t, t, acc);
        }
        if (acc < bd) {  // c increases along the loop: ties keep the lower index
            bd = acc;
            bc = c;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const float od = __shfl_xor_sync(0xffffffffu, bd, off);
        const int32_t oc = __shfl_xor_sync(0xffffffffu, bc, off);
        if (od < bd || (od == bd && oc < bc)) {
            bd = od;
            bc = oc;
        }
    }
    *best_d = bd;
    return bc;
}

// CUDA-core assignment of rows list[0..*count) (list == nullptr: all rows,
// count == nullptr: n). Centroids staged in shared memory with row stride
// d + 1 (bank-conflict free) when smem_c is set.
__global__ void km_assign_kernel(const float *F, int32_t n, int32_t d, const float *C, int32_t k,
                                 const int32_t *list, const int32_t *count, int32_t *labels, int32_t *changed,
                                 int smem_c) {
    extern __shared__ float s_c[];
    const float *cs = C;
    int32_t ldc = d;
    if (smem_c) {
        for (int64_t t = threadIdx.x; t < (int64_t)k * d; t += blockDim.x) s_c[(t / d) * (d + 1) + t % d] = C[t];
        __syncthreads();
        cs = s_c;
        ldc = d + 1;
    }
    const int64_t total = list ? (int64_t)*count : (int64_t)n;
    const int lane = threadIdx.x & 31;
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < total;
         w += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int32_t i = list ? list[w] : (int32_t)w;
        float bd;
        const int32_t c = km_decide_row(F + (int64_t)i * d, cs, ldc, k, d, &bd);
        if (lane == 0) {
            if (labels[i] != c) *changed = 1;
            labels[i] = c;
        }
    }
}

// The same exact decision, register-blocked for k <= 128 and d <= 256: a block
// of 128 threads takes 32 rows at a time; thread (g, h) = (t / 16, t % 16)
// scores rows 4g .. 4g + 3 against centroids h, h + 16, ..., h + 112, each
// pair an FP32 fused-multiply-add chain in index order (the same arithmetic
// as km_decide_row), with rows and centroids staged in shared memory (row
// stride d + 1: no bank conflicts). The 16 lanes of a row group then keep the
// smallest score, ties to the lowest centroid.
constexpr int kExRows = 32;
// Row stride of the staged rows: d + 1 (scalar loads, no bank conflicts), or
// d + 4 with 16-byte loads when d is a multiple of 4.
__host__ __device__ constexpr int ex_ld(int d, bool v4) { return v4 ? d + 4 : d + 1; }

template <bool V4>
__global__ void __launch_bounds__(128) km_assign_blocked_kernel(const float *F, int32_t n, int32_t d, const float *C,
                                                                int32_t k, const int32_t *list, const int32_t *count,
                                                                int32_t *labels, int32_t *changed) {
    extern __shared__ __align__(16) float s_ex[];
    const int ld = ex_ld(d, V4);
    float *sC = s_ex;                // [128][ld], rows >= k zero
    float *sF = s_ex + 128 * ld;     // [32][ld]
    for (int t = threadIdx.x; t < 128 * d; t += blockDim.x) {
        const int c = t / d, j = t % d;
        sC[c * ld + j] = (c < k) ? C[(int64_t)c * d + j] : 0.0f;
    }
    const int64_t total = list ? (int64_t)*count : (int64_t)n;
    const int g = threadIdx.x >> 4, h = threadIdx.x & 15;
    for (int64_t r0 = (int64_t)blockIdx.x * kExRows; r0 < total; r0 += (int64_t)gridDim.x * kExRows) {
        __syncthreads();  // sC ready (first pass) / sF free
        for (int t = threadIdx.x; t < kExRows * d; t += blockDim.x) {
            const int r = t / d, j = t % d;
            float v = 0.0f;
            if (r0 + r < total) {
                const int64_t i = list ? list[r0 + r] : r0 + r;
                v = F[i * d + j];
            }
            sF[r * ld + j] = v;
        }
        __syncthreads();
        float acc[4][8];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int m = 0; m < 8; ++m) acc[r][m] = 0.0f;
        const float *fr = sF + (4 * g) * ld;
        const float *cr = sC + h * ld;
        if (V4) {
            for (int j = 0; j < d; j += 4) {  // four columns per load, still added in index order
                float4 fv[4], cv[8];
#pragma unroll
                for (int r = 0; r < 4; ++r) fv[r] = *reinterpret_cast<const float4 *>(fr + r * ld + j);
#pragma unroll
                for (int m = 0; m < 8; ++m) cv[m] = *reinterpret_cast<const float4 *>(cr + (16 * m) * ld + j);
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int m = 0; m < 8; ++m) {
                        float t = __fsub_rn(fv[r].x, cv[m].x);
                        acc[r][m] = __fmaf_rn(t, t, acc[r][m]);
                        t = __fsub_rn(fv[r].y, cv[m].y);
                        acc[r][m] = __fmaf_rn(t, t, acc[r][m]);
                        t = __fsub_rn(fv[r].z, cv[m].z);
                        acc[r][m] = __fmaf_rn(t, t, acc[r][m]);
                        t = __fsub_rn(fv[r].w, cv[m].w);
                        acc[r][m] = __fmaf_rn(t, t, acc[r][m]);
                    }
            }
        } else {
            for (int j = 0; j < d; ++j) {
                float fv[4], cv[8];
#pragma unroll
                for (int r = 0; r < 4; ++r) fv[r] = fr[r * ld + j];
#pragma unroll
                for (int m = 0; m < 8; ++m) cv[m] = cr[(16 * m) * ld + j];
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int m = 0; m < 8; ++m) {
                        const float t = __fsub_rn(fv[r], cv[m]);
                        acc[r][m] = __fmaf_rn(t, t, acc[r][m]);
                    }
            }
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            float bd = INFINITY;
            int32_t bc = 0x7fffffff;
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                const int c = h + 16 * m;
                if (c < k && acc[r][m] < bd) {
                    bd = acc[r][m];
                    bc = c;
                }
            }
#pragma unroll
            for (int off = 1; off < 16; off <<= 1) {  // the 16 lanes of this row group
                const float od = __shfl_xor_sync(0xffffffffu, bd, off);
                const int32_t oc = __shfl_xor_sync(0xffffffffu, bc, off);
                if (od < bd || (od == bd && oc < bc)) {
                    bd = od;
                    bc = oc;
                }
            }
            const int64_t w = r0 + 4 * g + r;
            if (h == 0 && w < total) {
                const int64_t i = list ? list[w] : w;
                if (labels[i] != bc) *changed = 1;
                labels[i] = bc;
            }
        }
    }
}

// The exact decision for queued rows over their candidate centroids only
// (cmask bits, from the tensor-core pass): a warp per row, lanes over the
// candidates in increasing order, each an FP32 fused-multiply-add chain in
// index order; the smallest score wins, ties to the lowest centroid. Centroids
// staged in shared memory with row stride d + 1.
__global__ void km_assign_cands_kernel(const float *F, int32_t d, const float *C, int32_t k, const int32_t *list,
                                       const int32_t *count, const uint32_t *cmask, int32_t *labels,
                                       int32_t *changed) {
    extern __shared__ float s_cc[];
    const int32_t ldc = d + 1;
    for (int64_t t = threadIdx.x; t < (int64_t)k * d; t += blockDim.x) s_cc[(t / d) * ldc + t % d] = C[t];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t total = (int64_t)*count;
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < total;
         w += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int32_t i = list[w];
        const uint4 m4 = *reinterpret_cast<const uint4 *>(cmask + w * 4);
        const uint32_t m[4] = {m4.x, m4.y, m4.z, m4.w};
        const int n0 = __popc(m[0]), n1 = __popc(m[1]), n2 = __popc(m[2]);
        const int ncand = n0 + n1 + n2 + __popc(m[3]);
        const float *f = F + (int64_t)i * d;
        float bd = INFINITY;
        int32_t bc = 0x7fffffff;
        for (int t = lane; t < ncand; t += 32) {  // the t-th candidate in increasing order
            int q = 0, rem = t;
            const int cnt[3] = {n0, n1, n2};
            while (q < 3 && rem >= cnt[q]) rem -= cnt[q++];
            uint32_t bits = m[q];
            for (int r = 0; r < rem; ++r) bits &= bits - 1u;
            const int c = q * 32 + (__ffs(bits) - 1);
            const float *cc = s_cc + (int64_t)c * ldc;
            float acc = 0.f;
            for (int j = 0; j < d; ++j) {
                const float tt = __fsub_rn(__ldg(f + j), cc[j]);
                acc = __fmaf_rn(tt, tt, acc);
            }
            if (acc < bd || (acc == bd && c < bc)) {
                bd = acc;
                bc = c;
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const float od = __shfl_xor_sync(0xffffffffu, bd, off);
            const int32_t oc = __shfl_xor_sync(0xffffffffu, bc, off);
            if (od < bd || (od == bd && oc < bc)) {
                bd = od;
                bc = oc;
            }
        }
        if (lane == 0) {
            if (labels[i] != bc) *changed = 1;
            labels[i] = bc;
        }
    }
}

// inertia partials: part[b] = sum (FP64) over this block's rows of
// d(f_i, c_label_i), the FP32 fused-multiply-add chain in index order. A
// lane owns a row; when t_smem is set (d <= 128) each warp stages tiles of 32
// rows in shared memory (row stride d + 1, eight rows' coalesced loads in
// flight at a time), and
// the centroids are staged once per block when c_smem is set. Rows are added in a fixed order
// (lanes, warps, then tiles), so the result is deterministic.
constexpr int kInWarps = 8;
constexpr int kInRowVals = 4;  // values of a staged row per lane: tiles are staged when d <= 32 kInRowVals
__global__ void __launch_bounds__(kInWarps * 32) km_inertia_kernel(const float *__restrict__ F, int32_t n, int32_t d,
                                                                   const float *__restrict__ C, int32_t k,
                                                                   const int32_t *__restrict__ labels, int32_t t_smem,
                                                                   int32_t c_smem, double *part) {
    extern __shared__ float km_in_smem[];
    __shared__ double s_red[kInWarps];
    const int ld = d + 1, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *s_c = km_in_smem;
    float *s_t = km_in_smem + (c_smem ? (int64_t)k * ld : 0) + (t_smem ? (int64_t)warp * 32 * ld : 0);
    if (c_smem)
        for (int64_t t = threadIdx.x; t < (int64_t)k * d; t += blockDim.x) s_c[(t / d) * ld + t % d] = C[t];
    __syncthreads();
    double acc = 0.0;
    for (int64_t r0 = ((int64_t)blockIdx.x * kInWarps + warp) * 32; r0 < n; r0 += (int64_t)gridDim.x * kInWarps * 32) {
        const int rows = (int)min((int64_t)32, n - r0);
        if (t_smem)
            for (int r8 = 0; r8 < rows; r8 += 8) {  // eight rows' loads in flight
                float v[8][kInRowVals];
#pragma unroll
                for (int rr = 0; rr < 8; ++rr)
#pragma unroll
                    for (int u = 0; u < kInRowVals; ++u) {
                        const int j = lane + 32 * u;
                        v[rr][u] = (r8 + rr < rows && j < d) ? F[(r0 + r8 + rr) * d + j] : 0.f;
                    }
#pragma unroll
                for (int rr = 0; rr < 8; ++rr)
#pragma unroll
                    for (int u = 0; u < kInRowVals; ++u) {
                        const int j = lane + 32 * u;
                        if (r8 + rr < rows && j < d) s_t[(r8 + rr) * ld + j] = v[rr][u];
                    }
            }
        __syncwarp();
        if (lane < rows) {
            const int32_t c = labels[r0 + lane];
            const float *f = t_smem ? s_t + lane * ld : F + (r0 + lane) * d;
            const float *cc = c_smem ? s_c + (int64_t)c * ld : C + (int64_t)c * d;
            float sum = 0.f;
            for (int j = 0; j < d; ++j) {
                const float t = __fsub_rn(f[j], cc[j]);
                sum = __fmaf_rn(t, t, sum);
            }
            acc += (double)sum;
        }
        __syncwarp();
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) s_red[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int w = 0; w < kInWarps; ++w) a += s_red[w];
        part[blockIdx.x] = a;
    }
}

// Fixed-point scale of the centroid sums: every |F_ij| <= B = fmax_bits as a
// float, and n < 2^nb, so with values rounded to integers of F_ij 2^sh every
// partial sum stays below n 2^e 2^sh <= 2^62 (B < 2^e).
__device__ __forceinline__ int km_fix_shift(int32_t fmax_bits, int32_t n) {
    const float B = __int_as_float(fmax_bits);
    if (!(B > 0.f)) return 0;
    int e = 0;
    frexpf(B, &e);
    // at most 187: then every value is a multiple of 2^-sh (B < 2^-126 when
    // the cap binds: all values subnormal, multiples of 2^-149)
    return min(62 - (32 - __clz(n)) - e, 187);
}

// Centroid sums of one tile of clusters [c0, c0 + kt) over one contiguous
// range of rows, in batches of br rows. The sums live in shared memory as
// 64-bit integers; column chunk q (128 columns) of cluster c belongs to warp
// (c nch + q) mod kFixWarps alone, which adds it without atomics: lane l
// takes columns 128 q + 4 l .. + 3, kept at cells 128 q + 32 u + l of the
// cluster (u = 0..3), so every shared access of a warp is conflict free.
// STAGED: each batch (a contiguous run of br d floats, d a multiple of 4) is
// copied into one of kFixStages shared buffers by the TMA engine, three
// batches ahead; otherwise rows are read from global memory. The block then
// adds its sums into S and its counts into cnt with 64-bit integer atomics:
// integer addition is associative, so S is the same in any order.
constexpr int kFixWarps = 32;
constexpr int kFixStages = 3;
constexpr int kFixBatch = 128;  // rows per batch at most (4 label registers per lane)
constexpr int64_t kFixSmemBytes = 227 * 1024 - 1024;  // dynamic shared memory of one block
constexpr int64_t kFixAccBytes = 160 * 1024;          // of which at most this for the sums of a cluster tile

// the first column chunk q of cluster c that warp w owns: (c nch + q) mod kFixWarps == w
static_assert((kFixWarps & (kFixWarps - 1)) == 0, "kFixWarps must be a power of two");
__device__ __forceinline__ int km_fix_first_chunk(int w, int32_t c, int nch) {
    return (w - c * nch) & (kFixWarps - 1);
}

// The fixed-point value of the float x with bits u: floor(x 2^sh), by
// integer operations alone (a 64-bit conversion would run on the FP64 pipe).
// |x| = m 2^(e - 150) with m the 24-bit significand (e = 1 and no implicit
// bit for subnormals); the signed significand placed at bit 39 and shifted
// right arithmetically by 189 - sh - e (>= 1 because |x| 2^sh < 2^62,
// clamped to 63) is floor(x 2^sh). base = 189 - sh.
__device__ __forceinline__ long long km_fix_value(uint32_t u, int base) {
    const int e = (int)((u >> 23) & 255u);
    const int32_t s = (int32_t)u >> 31;  // 0 or -1
    const int32_t hi = (int32_t)(((u << 7) & 0x3fffff80u) | (e ? 0x40000000u : 0u));  // (m << 39) >> 32
    const uint32_t amt = (uint32_t)min(base - max(e, 1), 63);
    long long r;
    asm("shr.s64 %0, %1, %2;" : "=l"(r) : "l"((long long)((hi ^ s) - s) << 32), "r"(amt));
    return r;
}

struct FixParams {
    const float *F;
    const int32_t *labels;
    int32_t n, d, k, kc, nb, br, dpad;  // dpad: cells per cluster (128 per column chunk)
    const int32_t *fmax_bits;
    unsigned long long *S, *cnt;
    int32_t *status;  // bit 0: a bounded wait gave up
};

template <bool STAGED>
__global__ void __launch_bounds__(kFixWarps * 32, 1) km_fixsum_kernel(FixParams P) {
    extern __shared__ __align__(16) unsigned char km_fix_smem[];
    __shared__ int32_t s_done[kFixStages];   // warps done with the stage's current batch
    __shared__ int32_t s_last[kFixStages];   // the last batch issued into the stage
    __shared__ int32_t s_abort;
    const int32_t d = P.d, br = P.br, dpad = P.dpad;
    const int32_t tile = blockIdx.x / P.nb, blk = blockIdx.x % P.nb;
    const int32_t c0 = tile * P.kc, kt = min(P.kc, P.k - c0);
    uint64_t *s_bar = reinterpret_cast<uint64_t *>(km_fix_smem);             // [kFixStages]
    float *s_f = reinterpret_cast<float *>(km_fix_smem + 16 * kFixStages);  // [kFixStages][br][d]
    const int32_t stage_floats = STAGED ? br * d : 0;
    unsigned long long *s_acc = reinterpret_cast<unsigned long long *>(s_f + kFixStages * stage_floats);  // [kt][dpad]
    unsigned long long *s_cnt = s_acc + kt * dpad;                                                       // [kt]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int32_t t = tid; t < kt * dpad + kt; t += blockDim.x) s_acc[t] = 0ull;
    const int base = 189 - km_fix_shift(*P.fmax_bits, P.n);
    const int64_t r0 = (int64_t)P.n * blk / P.nb, r1 = (int64_t)P.n * (blk + 1) / P.nb;
    const int32_t nbatch = (int32_t)((r1 - r0 + br - 1) / br);
    const int nch = (d + 127) >> 7;

    auto issue = [&](int32_t bt) {  // one thread: batch bt into stage bt mod kFixStages
        const int st = bt % kFixStages;
        const int64_t r = r0 + (int64_t)bt * br;
        const uint32_t bytes = (uint32_t)(min((int64_t)br, r1 - r) * d * 4);
        s_last[st] = bt;
        mbar_arrive_expect_tx(&s_bar[st], bytes);
        bulk_g2s(s_f + st * stage_floats, P.F + r * d, bytes, &s_bar[st]);
    };
    if (tid == 0) {
        s_abort = 0;
        for (int st = 0; st < kFixStages; ++st) {
            s_done[st] = 0;
            s_last[st] = -1;
        }
        if (STAGED) {
            for (int st = 0; st < kFixStages; ++st) mbar_init(&s_bar[st], 1);
            fence_mbar_init();
            for (int32_t bt = 0; bt < kFixStages && bt < nbatch; ++bt) issue(bt);
        }
    }
    __syncthreads();
    // Warps move through the batches independently: the last warp done with
    // a stage refills it, so a warp that owns more rows of one batch delays
    // the others only when it falls a whole ring of stages behind.
    int32_t lv[kFixBatch / 32], ln[kFixBatch / 32];  // labels of rows 32 g + lane of this batch and the next
    auto load_labels = [&](int32_t bt, int32_t (&dst)[kFixBatch / 32]) {
        const int64_t r = r0 + (int64_t)bt * br;
        const int32_t rows = bt < nbatch ? (int32_t)min((int64_t)br, r1 - r) : 0;
#pragma unroll
        for (int g = 0; g < kFixBatch / 32; ++g)
            dst[g] = (32 * g + lane < rows) ? __ldg(P.labels + r + 32 * g + lane) : -1;
    };
    load_labels(0, lv);
    for (int32_t bt = 0; bt < nbatch; ++bt) {
        const int64_t r = r0 + (int64_t)bt * br;
        load_labels(bt + 1, ln);  // in flight while this batch is added
        const float *rowbase = P.F + r * d;
        const int st = bt % kFixStages;
        if (STAGED) {
            const bool landed = mbar_wait_bounded(&s_bar[st], (uint32_t)(bt / kFixStages) & 1u);
            if (!__all_sync(0xffffffffu, landed) || *(volatile int32_t *)&s_abort) {
                if (lane == 0) s_abort = 1;
                break;
            }
            rowbase = s_f + st * stage_floats;
        }
#pragma unroll
        for (int g = 0; g < kFixBatch / 32; ++g) {
            const int32_t c = lv[g] - c0;  // rows past the batch carry label -1
            const bool own = lv[g] >= 0 && c >= 0 && c < kt && km_fix_first_chunk(warp, c, nch) < nch;
            for (uint32_t m = __ballot_sync(0xffffffffu, own); m; m &= m - 1u) {
                const int l = __ffs(m) - 1;
                const int32_t cl = __shfl_sync(0xffffffffu, c, l);
                const float *f = rowbase + (32 * g + l) * d;
                unsigned long long *acc = s_acc + cl * dpad;
                const int q0 = km_fix_first_chunk(warp, cl, nch);
                for (int q = q0; q < nch; q += kFixWarps) {
                    const int j0 = 128 * q + 4 * lane;
                    float x[4];
                    if (STAGED) {
                        if (j0 >= d) continue;  // d is a multiple of 4: all four columns or none
                        const float4 t = *reinterpret_cast<const float4 *>(f + j0);
                        x[0] = t.x;
                        x[1] = t.y;
                        x[2] = t.z;
                        x[3] = t.w;
                    } else {
#pragma unroll
                        for (int u = 0; u < 4; ++u) x[u] = (j0 + u < d) ? __ldg(f + j0 + u) : 0.f;
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        acc[128 * q + 32 * u + lane] += (unsigned long long)km_fix_value(__float_as_uint(x[u]), base);
                }
                if (q0 == 0 && lane == 0) s_cnt[cl] += 1ull;
            }
        }
#pragma unroll
        for (int g = 0; g < kFixBatch / 32; ++g) lv[g] = ln[g];
        if (STAGED) {
            __syncwarp();
            if (lane == 0) {
                __threadfence_block();
                if (atomicAdd(&s_done[st], 1) == kFixWarps - 1) {  // the last warp done with this batch
                    s_done[st] = 0;
                    __threadfence_block();
                    if (bt + kFixStages < nbatch) {
                        fence_proxy_async();
                        issue(bt + kFixStages);
                    }
                }
            }
        }
    }
    __syncthreads();
    if (STAGED && s_abort) {  // a copy never landed: report, wait (bounded) for the copies issued, leave
        if (tid == 0) {
            atomicOr(P.status, 1);
            for (int st = 0; st < kFixStages; ++st)
                if (s_last[st] >= 0) mbar_wait_bounded(&s_bar[st], (uint32_t)(s_last[st] / kFixStages) & 1u);
        }
        return;
    }
    for (int32_t t = tid; t < kt * d; t += blockDim.x) {  // cell of column j: 128 q + 32 u + l, j = 128 q + 4 l + u
        const int32_t c = t / d, j = t - c * d;
        const unsigned long long v = s_acc[c * dpad + (j & ~127) + 32 * (j & 3) + ((j & 127) >> 2)];
        if (v) atomicAdd(P.S + (int64_t)(c0 + c) * d + j, v);
    }
    for (int t = tid; t < kt; t += blockDim.x)
        if (s_cnt[t]) atomicAdd(P.cnt + c0 + t, s_cnt[t]);
}

// c_c = (float)((S_c 2^-sh) / count_c) in FP64; an empty cluster keeps c_c
__global__ void km_fix_centroid_kernel(int32_t n, int32_t d, int32_t k, const int32_t *fmax_bits,
                                       const unsigned long long *S, const unsigned long long *cnt, float *C) {
    const int sh = km_fix_shift(*fmax_bits, n);
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)k * d;
         t += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long m = cnt[t / d];
        if (m == 0) continue;
        C[t] = (float)(ldexp((double)(long long)S[t], -sh) / (double)m);
    }
}

// ------------------------------------------------------------ tensor cores

// 2-D tiled TMA load of box {32 FP32 columns, rows} at (x, y) into shared memory
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int32_t x, int32_t y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor (tcgen05): K-major operand, 128-byte
// swizzle, 8-row groups 1024 bytes apart, start address `addr` (16-byte units).
__device__ __forceinline__ uint64_t umma_desc_sw128(uint32_t addr) {
    uint64_t desc = 0;
    desc |= (uint64_t)((addr >> 4) & 0x3FFFu);         // start address
    desc |= (uint64_t)1u << 16;                         // leading byte offset (unused for this layout)
    desc |= (uint64_t)(1024u >> 4) << 32;               // stride byte offset: 8 rows x 128 B
    desc |= (uint64_t)1u << 46;                         // descriptor version
    desc |= (uint64_t)2u << 61;                         // 128-byte swizzle
    return desc;
}

// Instruction descriptor: D FP32, A and B TF32, both K-major, M = 128, N = nmma.
__host__ __device__ constexpr uint32_t umma_idesc_tf32(int nmma) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(nmma >> 3) << 17) | ((uint32_t)(kTcRows >> 4) << 24);
}

// x = hi + lo + r with hi = x rounded to TF32 (nearest, ties away from
// zero), lo = (x - hi) rounded to TF32 (x - hi is exact in FP32), so
// |r| <= 2^-11 |x - hi| <= 2^-22 |x|.
__device__ __forceinline__ void km_split1(float v, float &h, float &l) {
    uint32_t a, b;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(a) : "f"(v));
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(b) : "f"(__fsub_rn(v, __uint_as_float(a))));
    h = __uint_as_float(a);
    l = __uint_as_float(b);
}

// 16-byte loads and stores (four independent ones per thread in flight) when
// the three arrays are 16-byte aligned; the remainder one element at a time.
__global__ void km_split_tf32_kernel(const float *x, int64_t count, float *hi, float *lo) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
    const bool vec = (((uintptr_t)x | (uintptr_t)hi | (uintptr_t)lo) & 15u) == 0;
    const int64_t nv = vec ? count / 4 : 0;
    const float4 *x4 = reinterpret_cast<const float4 *>(x);
    float4 *h4 = reinterpret_cast<float4 *>(hi), *l4 = reinterpret_cast<float4 *>(lo);
    constexpr int U = 4;
    for (int64_t i0 = tid; i0 < nv; i0 += nth * U) {
        float4 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (i0 + u * nth < nv) v[u] = __ldcs(x4 + i0 + u * nth);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (i0 + u * nth >= nv) continue;
            float4 h, l;
            km_split1(v[u].x, h.x, l.x);
            km_split1(v[u].y, h.y, l.y);
            km_split1(v[u].z, h.z, l.z);
            km_split1(v[u].w, h.w, l.w);
            h4[i0 + u * nth] = h;
            l4[i0 + u * nth] = l;
        }
    }
    for (int64_t i = 4 * nv + tid; i < count; i += nth) km_split1(x[i], hi[i], lo[i]);
}

// D (TMEM, FP32) (+)= A B^T for one K = 8 step of TF32 operands (A: 128 rows, B: N rows, both K-major)
__device__ __forceinline__ void umma_tf32(uint32_t dcol, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dcol),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

struct TcParams {
    int32_t n, d, k, nmma, ncols;  // ncols: TMEM columns per accumulator (power of two >= 32)
    int32_t stages;                // split operands: A stages of one 32-column chunk (high and low parts)
    const float *cn2;              // [k]
    const float *cmax;             // [1]
    const float *fn;               // [n]
    int32_t *labels;
    int32_t *changed;
    int32_t *list;                 // rows left to the exact decision
    uint32_t *cmask;               // [list slot][4]: the centroids each queued row must still compare
    int32_t *count;
    int32_t *status;               // bit 0: a bounded wait gave up
};

constexpr uint32_t kTcPolls = 1u << 24;

__device__ __forceinline__ bool tc_wait(uint64_t *bar, uint32_t parity, volatile int *abort) {
    for (uint32_t it = 0; it < kTcPolls; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 1023u) == 1023u && *abort) return false;
    }
    *abort = 1;
    return false;
}

// Warp roles: 0 = TMA producer, 1 = TMEM owner and MMA issuer, 2..5 = epilogue
// (128 threads, one tile row each). B: the centroids (nmma x d, rows >= k
// zero-filled by the copy), resident; two TMEM accumulators of ncols columns
// so that tile t + 1 multiplies while tile t is read. A, single pass: two
// stages of a whole 128 x d tile. A, SPLIT (F and C each given as TF32 high
// and low parts, x = hi + lo + r with |r| <= 2^-22 |x|): P.stages stages of
// one 32-column chunk of both parts, and three MMAs per K step, hi.hi +
// hi.lo + lo.hi, into the same accumulator.
constexpr int kTcMaxStages = 3;
constexpr float kTcProdSingle = 0.0078125f;        // 2^-7: products of TF32-truncated operands
constexpr float kTcProdSplit = 2.44140625e-04f;    // 2^-12: split operands
constexpr uint32_t kTcChunk = (uint32_t)kTcRows * 128;  // bytes of one 32-column FP32 chunk of a tile
constexpr int kTcSmemMax = 227 * 1024 - 2048;           // dynamic shared memory of the kernel, static beside it

template <bool SPLIT>
__global__ void __launch_bounds__(192, 1)
    kmeans_tc_kernel(const __grid_constant__ CUtensorMap mapF, const __grid_constant__ CUtensorMap mapC,
                     const __grid_constant__ CUtensorMap mapFlo, const __grid_constant__ CUtensorMap mapClo,
                     const TcParams P) {
    extern __shared__ __align__(16) unsigned char km_smem[];
    __shared__ __align__(8) uint64_t s_full[kTcMaxStages], s_empty[kTcMaxStages], s_tfull[2], s_tempty[2], s_bfull;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    __shared__ float s_cn2[128];  // |c|^2, +inf for the padding columns
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // 1024-byte aligned base for the swizzled tiles
    unsigned char *base = km_smem + ((1024u - (smem_u32(km_smem) & 1023u)) & 1023u);
    const int atoms = P.d / 32;                     // 128-byte K-chunks
    const uint32_t a_bytes = (uint32_t)kTcRows * P.d * 4;
    const uint32_t b_atom = (uint32_t)P.nmma * 128;
    unsigned char *sB = base;
    unsigned char *sBlo = base + (uint32_t)atoms * b_atom;  // SPLIT only
    unsigned char *sA0 = base + (uint32_t)atoms * b_atom * (SPLIT ? 2u : 1u);
    const int stages = SPLIT ? P.stages : 2;
    const uint32_t stage_bytes = SPLIT ? 2u * kTcChunk : a_bytes;  // SPLIT: high chunk, then low chunk
    const int n_tiles = (P.n + kTcRows - 1) / kTcRows;

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(&s_full[s], 1);
            mbar_init(&s_empty[s], 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&s_tfull[s], 1);
            mbar_init(&s_tempty[s], 4);  // one arrival per epilogue warp
        }
        mbar_init(&s_bfull, 1);
        s_abort = 0;
        fence_mbar_init();
    }
    for (int c = threadIdx.x; c < 128; c += blockDim.x) s_cn2[c] = (c < P.k) ? P.cn2[c] : INFINITY;
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(2 * P.ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;
    volatile int *abort = &s_abort;

    if (warp == 0 && lane == 0) {
        // producer: the centroids once, then the A tiles (or tile chunks) through the stages
        mbar_arrive_expect_tx(&s_bfull, (uint32_t)atoms * b_atom * (SPLIT ? 2u : 1u));
        for (int a = 0; a < atoms; ++a) {
            tma_load_2d(sB + a * b_atom, &mapC, 32 * a, 0, &s_bfull);
            if (SPLIT) tma_load_2d(sBlo + a * b_atom, &mapClo, 32 * a, 0, &s_bfull);
        }
        int t = 0;  // stage uses so far
        bool go = true;
        for (int tile = blockIdx.x; go && tile < n_tiles; tile += gridDim.x) {
            for (int a = 0; a < (SPLIT ? atoms : 1); ++a, ++t) {
                const int s = t % stages;
                if (t >= stages && !tc_wait(&s_empty[s], (uint32_t)((t / stages) - 1) & 1u, abort)) {
                    go = false;
                    break;
                }
                unsigned char *dst = sA0 + (uint32_t)s * stage_bytes;
                mbar_arrive_expect_tx(&s_full[s], stage_bytes);
                if (SPLIT) {
                    tma_load_2d(dst, &mapF, 32 * a, tile * kTcRows, &s_full[s]);
                    tma_load_2d(dst + kTcChunk, &mapFlo, 32 * a, tile * kTcRows, &s_full[s]);
                } else {
                    for (int c = 0; c < atoms; ++c)
                        tma_load_2d(dst + (uint32_t)c * kTcChunk, &mapF, 32 * c, tile * kTcRows, &s_full[s]);
                }
            }
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        const uint32_t idesc = umma_idesc_tf32(P.nmma);
        bool ok = tc_wait(&s_bfull, 0, abort);
        int t = 0, tt = 0;  // stage uses, tiles
        for (int tile = blockIdx.x; ok && tile < n_tiles; tile += gridDim.x, ++tt) {
            const int sa = tt & 1;
            if (tt >= 2 && !tc_wait(&s_tempty[sa], (uint32_t)((tt >> 1) - 1) & 1u, abort)) break;
            const uint32_t dcol = tmem + (uint32_t)sa * P.ncols;
            for (int a = 0; a < (SPLIT ? atoms : 1); ++a, ++t) {
                const int s = t % stages;
                if (!tc_wait(&s_full[s], (uint32_t)(t / stages) & 1u, abort)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const unsigned char *sA = sA0 + (uint32_t)s * stage_bytes;
                // K = 8 TF32 per instruction: 32 bytes of a 128-byte row
                for (int kk = (SPLIT ? 4 * a : 0); kk < (SPLIT ? 4 * a + 4 : P.d / 8); ++kk) {
                    const int c = kk >> 2;  // the chunk of B (and of A in the single pass)
                    const uint32_t off = (uint32_t)(kk & 3) * 32;
                    const uint32_t a_hi = smem_u32(sA + (SPLIT ? 0u : (uint32_t)c * kTcChunk)) + off;
                    const uint64_t bhi = umma_desc_sw128(smem_u32(sB + (uint32_t)c * b_atom) + off);
                    umma_tf32(dcol, umma_desc_sw128(a_hi), bhi, idesc, kk > 0 ? 1u : 0u);
                    if (SPLIT) {
                        const uint64_t blo = umma_desc_sw128(smem_u32(sBlo + (uint32_t)c * b_atom) + off);
                        umma_tf32(dcol, umma_desc_sw128(a_hi), blo, idesc, 1u);
                        umma_tf32(dcol, umma_desc_sw128(a_hi + kTcChunk), bhi, idesc, 1u);
                    }
                }
                // the stage is free once these MMAs complete
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(&s_empty[s]))
                             : "memory");
            }
            if (!ok) break;
            // the accumulator is ready once every MMA of the tile completes
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&s_tfull[sa]))
                         : "memory");
        }
    } else if (warp >= 2) {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31
        const int q = warp & 3;
        const float cmax = *P.cmax;
        int t = 0;
        for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++t) {
            const int s = t & 1;
            if (!tc_wait(&s_tfull[s], (uint32_t)(t >> 1) & 1u, abort)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int64_t row = (int64_t)tile * kTcRows + q * 32 + lane;
            // the row's error margin first: the candidate test below needs it
            const float fi = row < P.n ? __ldg(P.fn + row) : 0.0f;
            const float prod = SPLIT ? kTcProdSplit : kTcProdSingle;
            const float two_e = 2.0f * (prod * fi * cmax + 1.52587890625e-05f * (fi + cmax) * (fi + cmax));
            // four interleaved best / second-best trackers (columns u % 4), branch-free; a column is a
            // candidate when e_c <= (its tracker's best so far) + 2 E_i: a superset of the centroids within
            // 2 E_i of the final best, since every tracker's best only decreases towards values >= it
            float t1[4], t2[4];
            int32_t tc[4];
            uint32_t cm0 = 0u, cm1 = 0u, cm2 = 0u, cm3 = 0u;
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                t1[v] = INFINITY;
                t2[v] = INFINITY;
                tc[v] = 0x7fffffff;
            }
            for (int c0 = 0; c0 < P.nmma; c0 += 32) {
                // two 16-column loads in flight, one wait
                uint32_t r[32];
                const uint32_t taddr = tmem + (uint32_t)s * P.ncols + (uint32_t)c0 + ((uint32_t)(q * 32) << 16);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                    "%13, %14, %15}, [%16];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                      "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                      "=r"(r[14]), "=r"(r[15])
                    : "r"(taddr));
                const bool two = c0 + 16 < P.nmma;
                if (two)
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
                        "%12, %13, %14, %15}, [%16];"
                        : "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
                          "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
                          "=r"(r[30]), "=r"(r[31])
                        : "r"(taddr + 16u));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                uint32_t wb = 0u;  // candidate bits of columns c0 .. c0 + 31
#pragma unroll
                for (int u = 0; u < 32; ++u) {
                    if (u < 16 || two) {
                        const int v = u & 3;
                        const float e = fmaf(-2.0f, __uint_as_float(r[u]), s_cn2[c0 + u]);  // +inf past k
                        const bool lt = e < t1[v];  // strict: the earlier (lower) column keeps ties
                        t2[v] = fminf(t2[v], fmaxf(t1[v], e));
                        tc[v] = lt ? c0 + u : tc[v];
                        t1[v] = fminf(t1[v], e);
                        wb |= (c0 + u < P.k && e <= t1[v] + two_e) ? (1u << u) : 0u;
                    }
                }
                if (c0 == 0) cm0 = wb;
                else if (c0 == 32) cm1 = wb;
                else if (c0 == 64) cm2 = wb;
                else cm3 = wb;
            }
            // the accumulator may be overwritten once every epilogue warp has read it
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&s_tempty[s]);
            // merge: smallest value, ties to the lowest column; second = the others' best or the winner's second
            int w = 0;
#pragma unroll
            for (int v = 1; v < 4; ++v)
                if (t1[v] < t1[w] || (t1[v] == t1[w] && tc[v] < tc[w])) w = v;
            const float b1 = t1[w];
            const int32_t c1 = tc[w];
            float b2 = t2[w];
#pragma unroll
            for (int v = 0; v < 4; ++v)
                if (v != w) b2 = fminf(b2, t1[v]);
            bool queue = false;
            if (row < P.n) {
                queue = P.k > 1 && !(b2 - b1 > two_e);
                if (!queue) {
                    if (P.labels[row] != c1) *P.changed = 1;
                    P.labels[row] = c1;
                }
            }
            const unsigned qm = __ballot_sync(0xffffffffu, queue);
            // one queue slot reservation per warp
            if (qm) {
                int32_t slot0 = 0;
                if (lane == 0) slot0 = atomicAdd(P.count, __popc(qm));
                slot0 = __shfl_sync(0xffffffffu, slot0, 0);
                if (queue) {
                    const int32_t slot = slot0 + __popc(qm & ((1u << lane) - 1u));
                    P.list[slot] = (int32_t)row;
                    *reinterpret_cast<uint4 *>(P.cmask + (int64_t)slot * 4) = make_uint4(cm0, cm1, cm2, cm3);
                }
            }
        }
    }
    // teardown: every role has left its loop
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0 && s_abort) atomicOr(P.status, 1);
    if (warp == 1) {
        __syncwarp();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * P.ncols)
                     : "memory");
    }
}

// ------------------------------------------------------------ host
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static sf_status encode_fn(EncodeTiledFn *out) {
    static EncodeTiledFn fn = nullptr;
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p) {
            cudaGetLastError();
            set_error("cuTensorMapEncodeTiled is not available from the driver");
            return SF_ERR_CUDA;
        }
        fn = (EncodeTiledFn)p;
    }
    *out = fn;
    return SF_OK;
}

// FP32 row-major [rows][d] with 128-byte swizzled boxes of {32, box_rows}
static sf_status encode_rows(CUtensorMap *map, const float *ptr, int64_t rows, int32_t d, int32_t box_rows) {
    EncodeTiledFn fn;
    sf_status st = encode_fn(&fn);
    if (st) return st;
    cuuint64_t dims[2] = {(cuuint64_t)d, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)d * 4};
    cuuint32_t box[2] = {32, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(ptr), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
        return SF_ERR_CUDA;
    }
    return SF_OK;
}

// Pinned host words that the iterations' flags are copied into without
// blocking: one buffer per host thread (calls from one thread run one after
// another), grown when a call needs more. It is never freed (a few hundred
// bytes per thread; freeing it while the CUDA runtime shuts down at exit is
// not safe).
static sf_status host_flags(int32_t **out, size_t count) {
    struct Buf {
        int32_t *p = nullptr;
        size_t n = 0;
    };
    static thread_local Buf buf;
    if (buf.n < count) {
        if (buf.p) cudaFreeHost(buf.p);
        buf.p = nullptr;
        buf.n = 0;
        void *q = nullptr;
        const size_t want = count < 64 ? 64 : count;
        const cudaError_t e = cudaHostAlloc(&q, want * sizeof(int32_t), cudaHostAllocPortable);
        if (e != cudaSuccess) return cuda_fail(e, "cudaHostAlloc (k-means flags)");
        buf.p = static_cast<int32_t *>(q);
        buf.n = want;
    }
    *out = buf.p;
    return SF_OK;
}

static bool tc_shape_ok(int32_t d, int32_t k) { return d % 32 == 0 && d >= 32 && d <= 128 && k >= 1 && k <= 128; }

static int tc_smem_bytes(int32_t d, int32_t nmma) {
    return 1024 /* alignment slack */ + (d / 32) * nmma * 128 + 2 * kTcRows * d * 4;
}

}  // namespace sf

using namespace sf;

extern "C" SF_API sf_status sf_kmeans(const float *F, int32_t n, int32_t d, int32_t k, float *C, int32_t max_iter,
                                      int32_t mode, int32_t *labels, int32_t *iters, double *inertia,
                                      void *stream) {
    SF_ARG(F && C && labels && iters, "F/C/labels/iters is NULL");
    SF_ARG(n >= 1 && d >= 1 && d <= 4096, "need n >= 1 and 1 <= d <= 4096");
    SF_ARG(k >= 1 && k <= 1023, "k must be in [1, 1023]");
    SF_ARG(max_iter >= 1, "max_iter must be >= 1");
    SF_ARG(mode == SF_KMEANS_AUTO || mode == SF_KMEANS_TENSOR || mode == SF_KMEANS_CUDA_CORES ||
               mode == SF_KMEANS_TENSOR_SINGLE,
           "mode must be SF_KMEANS_*");
    const bool aligned = ((uintptr_t)F % 16 == 0) && ((uintptr_t)C % 16 == 0);
    const bool tc = mode != SF_KMEANS_CUDA_CORES && tc_shape_ok(d, k) && aligned;
    SF_ARG((mode != SF_KMEANS_TENSOR && mode != SF_KMEANS_TENSOR_SINGLE) || tc,
           "the tensor-core assignment needs d a multiple of 32 in [32, 128], k <= 128 and 16-byte aligned F and C");
    const bool split = tc && mode != SF_KMEANS_TENSOR_SINGLE;
    cudaStream_t s = (cudaStream_t)stream;
    Scratch sc(s);
    float *fn = nullptr, *cn2 = nullptr, *cmax = nullptr;
    uint32_t *cmask = nullptr;
    int32_t *changed = nullptr, *bad = nullptr, *list = nullptr, *count = nullptr, *fmax_bits = nullptr;
    unsigned long long *S = nullptr;  // [k][d] fixed-point sums, then [k] counts
    double *ipart = nullptr, *isum = nullptr;
    const int ig = 2 * sm_count();
    sf_status st;
    if ((st = sc.get(&fn, (size_t)n)) || (st = sc.get(&cn2, (size_t)k)) || (st = sc.get(&cmax, 1)) ||
        (st = sc.get(&changed, 2)) || (st = sc.get(&bad, 1)) || (st = sc.get(&list, (size_t)n)) ||
        (st = sc.get(&count, 2)) || (st = sc.get(&fmax_bits, 1)) || (st = sc.get(&S, (size_t)k * (d + 1))) ||
        (st = sc.get(&ipart, (size_t)ig)) || (st = sc.get(&isum, 1)))
        return st;
    SF_CHECK_CUDA(cudaMemsetAsync(labels, 0xff, sizeof(int32_t) * (size_t)n, s));  // -1: no label yet
    SF_CHECK_CUDA(cudaMemsetAsync(bad, 0, sizeof(int32_t), s));
    SF_CHECK_CUDA(cudaMemsetAsync(fmax_bits, 0, sizeof(int32_t), s));
    km_row_norm_kernel<<<4 * sm_count(), 256, 0, s>>>(F, n, d, fn, bad, fmax_bits);
    if ((st = check_launch("km_row_norm_kernel"))) return st;

    // tensor-core setup (split: F and C as TF32 high and low parts, F once, C every assignment)
    CUtensorMap mapF, mapC, mapFlo, mapClo;
    TcParams T = {};
    int tc_grid = 0, tc_smem = 0;
    float *Fhi = nullptr, *Flo = nullptr, *Chi = nullptr, *Clo = nullptr;
    if (tc) {
        const int nmma = (k + 15) / 16 * 16;
        int ncols = 32;
        while (ncols < nmma) ncols *= 2;
        if (split) {
            if ((st = sc.get(&Fhi, (size_t)n * d)) || (st = sc.get(&Flo, (size_t)n * d)) ||
                (st = sc.get(&Chi, (size_t)k * d)) || (st = sc.get(&Clo, (size_t)k * d)))
                return st;
            km_split_tf32_kernel<<<8 * sm_count(), 256, 0, s>>>(F, (int64_t)n * d, Fhi, Flo);
            if ((st = check_launch("km_split_tf32_kernel"))) return st;
            if ((st = encode_rows(&mapF, Fhi, n, d, kTcRows)) || (st = encode_rows(&mapFlo, Flo, n, d, kTcRows)) ||
                (st = encode_rows(&mapC, Chi, k, d, nmma)) || (st = encode_rows(&mapClo, Clo, k, d, nmma)))
                return st;
            const int fixed = 1024 + 2 * (d / 32) * nmma * 128;
            T.stages = fixed + kTcMaxStages * 2 * (int)kTcChunk <= kTcSmemMax ? kTcMaxStages : 2;
            tc_smem = fixed + T.stages * 2 * (int)kTcChunk;
        } else {
            if ((st = encode_rows(&mapF, F, n, d, kTcRows)) || (st = encode_rows(&mapC, C, k, d, nmma))) return st;
            mapFlo = mapF;
            mapClo = mapC;
            tc_smem = tc_smem_bytes(d, nmma);
        }
        SF_CHECK_CUDA(cudaFuncSetAttribute(split ? (const void *)kmeans_tc_kernel<true>
                                                 : (const void *)kmeans_tc_kernel<false>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem));
        SF_CHECK_CUDA(cudaFuncSetAttribute(km_assign_cands_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)((size_t)k * (d + 1) * sizeof(float))));
        const int n_tiles = (n + kTcRows - 1) / kTcRows;
        tc_grid = n_tiles < sm_count() ? n_tiles : sm_count();
        T.n = n;
        T.d = d;
        T.k = k;
        T.nmma = nmma;
        T.ncols = ncols;
        T.cn2 = cn2;
        T.cmax = cmax;
        T.fn = fn;
        T.labels = labels;
        T.changed = changed;
        T.list = list;
        T.count = count;
        if ((st = sc.get(&cmask, (size_t)n * 4))) return st;
        T.cmask = cmask;
        T.status = device_status();
        SF_ARG(T.status, "device status word unavailable");
    }
    // CUDA-core assignment of every row: register-blocked for k <= 128 and d <= 256, else a warp per row
    // with the centroids in shared memory when they fit
    const bool blocked = k <= 128 && d <= 256;
    const bool ex_v4 = d % 4 == 0;
    const size_t ex_smem = (size_t)(128 + kExRows) * ex_ld(d, ex_v4) * sizeof(float);
    const void *ex_fn =
        ex_v4 ? (const void *)km_assign_blocked_kernel<true> : (const void *)km_assign_blocked_kernel<false>;
    const size_t c_smem = (size_t)k * (d + 1) * sizeof(float);
    const int smem_c = c_smem <= 160 * 1024 ? 1 : 0;
    int ex_occ = 1;
    if (!tc && blocked) {
        SF_CHECK_CUDA(cudaFuncSetAttribute(ex_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ex_smem));
        SF_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ex_occ, ex_fn, 128, ex_smem));
    } else if (!tc && smem_c) {
        SF_CHECK_CUDA(cudaFuncSetAttribute(km_assign_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)c_smem));
    }
    const int assign_grid = blocked ? (ex_occ > 0 ? ex_occ : 1) * sm_count() : (smem_c ? sm_count() : 4 * sm_count());
    auto exact = [&](const int32_t *lst, const int32_t *cnt, int32_t *chg) -> sf_status {
        if (blocked && ex_v4)
            km_assign_blocked_kernel<true><<<assign_grid, 128, ex_smem, s>>>(F, n, d, C, k, lst, cnt, labels, chg);
        else if (blocked)
            km_assign_blocked_kernel<false><<<assign_grid, 128, ex_smem, s>>>(F, n, d, C, k, lst, cnt, labels, chg);
        else
            km_assign_kernel<<<assign_grid, 256, smem_c ? c_smem : 0, s>>>(F, n, d, C, k, lst, cnt, labels, chg,
                                                                           smem_c);
        return check_launch("km_assign_kernel");
    };

    // update layout: tiles of FP.kc clusters whose sums fit in shared memory beside the row stages
    FixParams FP = {};
    size_t fix_smem = 0;
    unsigned fix_grid = 0;
    const void *fix_fn = nullptr;
    {
        const bool staged = d % 4 == 0 && (uintptr_t)F % 16 == 0;
        const int32_t dpad = (d + 127) / 128 * 128;
        const int64_t cell = 8 * (int64_t)dpad + 8;
        const int64_t kc = std::max<int64_t>(1, std::min<int64_t>(k, kFixAccBytes / cell));
        const int64_t ntile = (k + kc - 1) / kc;
        FP.kc = (int32_t)((k + ntile - 1) / ntile);
        const int64_t acc = (int64_t)FP.kc * cell;
        const int64_t head = 16 * kFixStages;
        int64_t br = kFixBatch;
        if (staged) br = std::min<int64_t>(kFixBatch, (kFixSmemBytes - head - acc) / ((int64_t)kFixStages * 4 * d));
        SF_ARG(br >= 1, "k-means: centroid sums do not fit in shared memory");
        fix_smem = (size_t)(head + (staged ? (int64_t)kFixStages * br * 4 * d : 0) + acc);
        fix_fn = staged ? (const void *)km_fixsum_kernel<true> : (const void *)km_fixsum_kernel<false>;
        SF_CHECK_CUDA(cudaFuncSetAttribute(fix_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fix_smem));
        int occ = 0;
        SF_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fix_fn, kFixWarps * 32, fix_smem));
        FP.nb = (int32_t)std::max<int64_t>(1, std::min<int64_t>(n, (int64_t)std::max(occ, 1) * sm_count() / ntile));
        fix_grid = (unsigned)(ntile * FP.nb);
        FP.F = F;
        FP.labels = labels;
        FP.n = n;
        FP.d = d;
        FP.k = k;
        FP.br = (int32_t)br;
        FP.dpad = dpad;
        FP.fmax_bits = fmax_bits;
        FP.S = S;
        FP.cnt = S + (size_t)k * d;
        FP.status = device_status();
        SF_ARG(FP.status, "device status word unavailable");
    }
    // inertia: tiles of 32 rows per warp in shared memory, the centroids too when they fit
    const int in_t_smem = d <= 32 * kInRowVals ? 1 : 0;
    const size_t in_tiles = in_t_smem ? (size_t)kInWarps * 32 * (d + 1) * sizeof(float) : 0;
    const size_t in_cent = (size_t)k * (d + 1) * sizeof(float);
    const int in_c_smem = in_tiles + in_cent <= (size_t)kFixSmemBytes ? 1 : 0;
    const size_t in_smem = in_tiles + (in_c_smem ? in_cent : 0);
    int in_grid = 1;
    if (inertia) {
        SF_CHECK_CUDA(
            cudaFuncSetAttribute(km_inertia_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)in_smem));
        int occ = 0;
        SF_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, km_inertia_kernel, kInWarps * 32, in_smem));
        in_grid = std::min(ig, std::max(occ, 1) * sm_count());
    }
    // Lloyd iterations with one assignment of look-ahead: assignment t and its flags' copy to the host are
    // queued, then the host waits for assignment t - 1's flags (the GPU meanwhile runs update t - 1 and
    // assignment t), so the GPU does not idle on the host round trip. An update queued after an assignment
    // that turns out to have changed no label recomputes the same centroids bit for bit (the same labels,
    // the same exact sums), and the assignment after it the same labels: the look-ahead leaves labels,
    // centroids, inertia and the iteration count as a loop that waits after every assignment.
    // flags of assignment t in slot t & 1 (device: changed; pinned host: changed, bad): at most two assignments
    // are in flight, and a slot is cleared for assignment t only after the host has read assignment t - 2
    int32_t *hflags = nullptr;
    if ((st = host_flags(&hflags, 4))) return st;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    SF_CHECK_CUDA(cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming));
    if (cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming) != cudaSuccess) {
        cudaEventDestroy(ev[0]);
        return cuda_fail(cudaGetLastError(), "cudaEventCreate");
    }
    struct EvGuard {
        cudaEvent_t *e;
        ~EvGuard() {
            cudaEventDestroy(e[0]);
            cudaEventDestroy(e[1]);
        }
    } ev_guard{ev};
    auto assign = [&](int t) -> sf_status {
        sf_status r;
        SF_CHECK_CUDA(cudaMemsetAsync(changed + (t & 1), 0, sizeof(int32_t), s));
        km_centroid_norm_kernel<<<1, 1024, 0, s>>>(C, k, d, cn2, cmax, bad);
        if ((r = check_launch("km_centroid_norm_kernel"))) return r;
        if (tc) {
            SF_CHECK_CUDA(cudaMemsetAsync(count, 0, sizeof(int32_t), s));
            cudaEvent_t ea = nullptr, eb = nullptr;
            const bool prof = profiling_on() && profile_events(&ea, &eb);
            if (split) {
                km_split_tf32_kernel<<<sm_count(), 256, 0, s>>>(C, (int64_t)k * d, Chi, Clo);
                if ((r = check_launch("km_split_tf32_kernel"))) return r;
            }
            TcParams Tt = T;
            Tt.changed = changed + (t & 1);
            if (prof) cudaEventRecord(ea, s);
            if (split) kmeans_tc_kernel<true><<<tc_grid, 192, tc_smem, s>>>(mapF, mapC, mapFlo, mapClo, Tt);
            else kmeans_tc_kernel<false><<<tc_grid, 192, tc_smem, s>>>(mapF, mapC, mapFlo, mapClo, Tt);
            if ((r = check_launch("kmeans_tc_kernel"))) return r;
            if (prof) {
                cudaEventRecord(eb, s);
                // compulsory bytes: the rows once, the centroids per CTA (each in two parts when split),
                // labels read and written
                const double parts = split ? 2.0 : 1.0;
                profile_record(ea, eb, parts * ((double)n * d * 4 + (double)tc_grid * k * d * 4) + (double)n * 8,
                               kProfTagKmeansTc);
            }
            km_assign_cands_kernel<<<4 * sm_count(), 256, (size_t)k * (d + 1) * sizeof(float), s>>>(
                F, d, C, k, list, count, cmask, labels, changed + (t & 1));
            if ((r = check_launch("km_assign_cands_kernel"))) return r;
        } else if ((r = exact(nullptr, nullptr, changed + (t & 1)))) {
            return r;
        }
        SF_CHECK_CUDA(cudaMemcpyAsync(hflags + 2 * (t & 1), changed + (t & 1), sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        SF_CHECK_CUDA(cudaMemcpyAsync(hflags + 2 * (t & 1) + 1, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        SF_CHECK_CUDA(cudaEventRecord(ev[t & 1], s));
        return SF_OK;
    };
    auto update = [&]() -> sf_status {
        // exact fixed-point sums per cluster, then the FP64 means
        sf_status r;
        SF_CHECK_CUDA(cudaMemsetAsync(S, 0, sizeof(unsigned long long) * (size_t)k * (d + 1), s));
        if (fix_fn == (const void *)km_fixsum_kernel<true>)
            km_fixsum_kernel<true><<<fix_grid, kFixWarps * 32, fix_smem, s>>>(FP);
        else
            km_fixsum_kernel<false><<<fix_grid, kFixWarps * 32, fix_smem, s>>>(FP);
        if ((r = check_launch("km_fixsum_kernel"))) return r;
        km_fix_centroid_kernel<<<(k * d + 255) / 256, 256, 0, s>>>(n, d, k, fmax_bits, S, S + (size_t)k * d, C);
        return check_launch("km_fix_centroid_kernel");
    };
    // assignment t's flags on the host (its event has completed): SF_ERR_NUMERIC for a non-finite row or
    // centroid; *conv: no label changed (from the second assignment on)
    auto landed = [&](int t, bool *conv) -> sf_status {
        SF_CHECK_CUDA(cudaEventSynchronize(ev[t & 1]));
        if (hflags[2 * (t & 1) + 1]) {
            set_error("non-finite feature row or centroid");
            return SF_ERR_NUMERIC;
        }
        *conv = t >= 1 && hflags[2 * (t & 1)] == 0;
        return SF_OK;
    };
    int final_t = -1;
    bool conv_final = false;
    for (int t = 0; t < max_iter; ++t) {
        if ((st = assign(t))) return st;
        if (t >= 1) {
            bool conv = false;
            if ((st = landed(t - 1, &conv))) return st;
            if (conv) {  // assignment t - 1 changed nothing: update t - 1 and assignment t were no-ops
                final_t = t - 1;
                conv_final = true;
                break;
            }
        }
        if (t == max_iter - 1) {
            bool conv = false;
            if ((st = landed(t, &conv))) return st;
            final_t = t;
            conv_final = conv;
            break;
        }
        if ((st = update())) return st;
    }
    SF_CHECK_CUDA(cudaStreamSynchronize(s));
    if ((st = sf_device_check(stream))) return st;
    if (inertia) {  // of the final labels and the centroids they were assigned to
        km_inertia_kernel<<<in_grid, kInWarps * 32, in_smem, s>>>(F, n, d, C, k, labels, in_t_smem, in_c_smem, ipart);
        if ((st = check_launch("km_inertia_kernel"))) return st;
        if ((st = reduce_sum_f64(ipart, in_grid, isum, s))) return st;
        SF_CHECK_CUDA(cudaMemcpyAsync(inertia, isum, sizeof(double), cudaMemcpyDeviceToHost, s));
        SF_CHECK_CUDA(cudaStreamSynchronize(s));
    }
    if (!conv_final && (st = update())) return st;  // the last assignment changed labels: its update
    *iters = final_t + 1;
    return SF_OK;
}
