// Diagnostics: the gather ceiling (sf_gather_ceiling), the sweep kernel's
// random-row data movement alone, timed on synthetic data, as the practical
// ceiling its launches are compared with; and the self-test of the bounded
// waits (sf_selftest_bounded_wait).
#include <math.h>

#include "sf_step.cuh"

namespace sf {

__device__ __forceinline__ uint64_t probe_mix(uint64_t z) {
    // SplitMix64 finaliser (Steele, Lea, Flood, OOPSLA 2014)
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// table: hashed BF16 values in [-0.5, 0.5), last row zero
__global__ void probe_fill_table(uint16_t *T, int64_t rows, int32_t cols) {
    const int64_t total = rows * cols;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const float v = (t / cols == rows - 1) ? 0.0f : (float)(probe_mix((uint64_t)t) & 0xffff) / 65536.0f - 0.5f;
        T[t] = (uint16_t)(__float_as_uint(v) >> 16);
    }
}

__global__ void probe_fill_idx(int32_t *idx, int64_t count, int64_t n) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x)
        idx[t] = (int32_t)(probe_mix((uint64_t)t + 0x5851F42D4C957F2Dull) % (uint64_t)n);
}

__device__ __forceinline__ void probe_add(float (&acc)[8], const uint4 v) {
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        acc[2 * i] += __uint_as_float(w[i] << 16);
        acc[2 * i + 1] += __uint_as_float(w[i] & 0xffff0000u);
    }
}

// WROW: each output row's FP32 sums written back (as a sweep writes T_j);
// else one float per row (the gathers alone).
template <int LPR, bool WROW>
__global__ void __launch_bounds__(256, 4) probe_gather_kernel(const uint16_t *T, const int32_t *idx, int64_t n_out,
                                                              int32_t deg, float *out) {
    constexpr int COLS = LPR * 8;  // BF16 columns per row
    constexpr int RPB = 256 / LPR;
    const int q = threadIdx.x % LPR, grp = threadIdx.x / LPR;
    for (int64_t row = (int64_t)blockIdx.x * RPB + grp; row < n_out; row += (int64_t)gridDim.x * RPB) {
        const int32_t *ip = idx + row * deg;
        float acc[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) acc[v] = 0.f;
        int32_t j = 0;
        for (; j + 8 <= deg; j += 8) {
            const int4 a = __ldg(reinterpret_cast<const int4 *>(ip + j));
            const int4 b = __ldg(reinterpret_cast<const int4 *>(ip + j + 4));
            const int32_t k[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
            uint4 x[8];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                x[u] = __ldg(reinterpret_cast<const uint4 *>(T + (int64_t)k[u] * COLS + q * 8));
#pragma unroll
            for (int u = 0; u < 8; ++u) probe_add(acc, x[u]);
        }
        if (j < deg) {  // deg is a multiple of 4
            const int4 a = __ldg(reinterpret_cast<const int4 *>(ip + j));
            const int32_t k[4] = {a.x, a.y, a.z, a.w};
            uint4 x[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                x[u] = __ldg(reinterpret_cast<const uint4 *>(T + (int64_t)k[u] * COLS + q * 8));
#pragma unroll
            for (int u = 0; u < 4; ++u) probe_add(acc, x[u]);
        }
        if (WROW) {
            float4 *o = reinterpret_cast<float4 *>(out + row * COLS + q * 8);
            __stcs(o, make_float4(acc[0], acc[1], acc[2], acc[3]));
            __stcs(o + 1, make_float4(acc[4], acc[5], acc[6], acc[7]));
        } else {
            float t = 0.f;
#pragma unroll
            for (int v = 0; v < 8; ++v) t += acc[v];
            if (q == 0) out[row] = t;
        }
    }
}

template <int LPR>
static void probe_launch(int grid, cudaStream_t s, const uint16_t *T, const int32_t *idx, int64_t n, int32_t deg,
                         float *out, bool write_rows) {
    if (write_rows) probe_gather_kernel<LPR, true><<<grid, 256, 0, s>>>(T, idx, n, deg, out);
    else probe_gather_kernel<LPR, false><<<grid, 256, 0, s>>>(T, idx, n, deg, out);
}

// One block waits on an mbarrier that nothing ever completes, with the same
// try-wait the sweep kernels use, gives up after `polls` polls and sets the
// device status word as a sweep kernel whose staged copy never landed would.
__global__ void selftest_wait_kernel(int32_t polls, int32_t *status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    bool landed = false;
    for (int32_t i = 0; i < polls && !landed; ++i) landed = mbar_try_wait(&bar, 0);
    if (!landed && threadIdx.x == 0) atomicOr(status, 1);
}

// One thread waits, as a persistent batch tile does, for a graph whose arrival
// counter nothing increments (step 1 of a graph with one chunk), gives up after
// `polls` polls and sets the status word and the abort flag as the batch
// kernel does.
__global__ void selftest_arrival_kernel(int32_t polls, int32_t *status, uint32_t *counters, int32_t *tables) {
    BatchSched S = {};
    S.n_tiles = 1;
    S.chunk = 1;
    S.n_chunks = 1;
    S.p = 2;
    S.chunk_glo = tables;       // chunk 0 covers graph 0 ...
    S.chunk_ghi = tables;
    S.graph_chunks = counters;  // ... which has one chunk
    S.done = counters + 1;      // and has completed nothing
    S.abort = tables + 1;
    if (!wait_graph_deps(S, 1, 0, (uint32_t)polls)) {
        atomicOr(status, 2);
        atomicExch(S.abort, 1);
    }
}

}  // namespace sf

using namespace sf;

extern "C" SF_API sf_status sf_selftest_arrival_wait(int32_t polls, void *stream) {
    SF_ARG(polls >= 1 && polls <= (1 << 16), "polls must be in [1, 2^16]");
    int32_t *status = device_status();
    SF_ARG(status, "device status word unavailable");
    cudaStream_t s = (cudaStream_t)stream;
    Scratch sc(s);
    uint32_t *counters = nullptr;
    int32_t *tables = nullptr;
    sf_status st;
    if ((st = sc.get(&counters, 2)) || (st = sc.get(&tables, 2))) return st;
    const uint32_t c_h[2] = {1u, 0u};  // graph 0: one chunk, nothing completed
    const int32_t t_h[2] = {0, 0};     // chunk 0 covers graph 0; abort flag clear
    SF_CHECK_CUDA(cudaMemcpyAsync(counters, c_h, sizeof(c_h), cudaMemcpyHostToDevice, s));
    SF_CHECK_CUDA(cudaMemcpyAsync(tables, t_h, sizeof(t_h), cudaMemcpyHostToDevice, s));
    selftest_arrival_kernel<<<1, 1, 0, s>>>(polls, status, counters, tables);
    st = check_launch("selftest_arrival_kernel");
    SF_CHECK_CUDA(cudaStreamSynchronize(s));  // the host copies and the scratch outlive the kernel
    return st;
}

extern "C" SF_API sf_status sf_selftest_bounded_wait(int32_t polls, void *stream) {
    SF_ARG(polls >= 1 && polls <= (1 << 20), "polls must be in [1, 2^20]");
    int32_t *status = device_status();
    SF_ARG(status, "device status word unavailable");
    selftest_wait_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(polls, status);
    return check_launch("selftest_wait_kernel");
}

static sf_status gather_rate(int64_t n_rows, int32_t row_bytes, int32_t deg, int32_t reps, bool write_rows,
                             void *stream, double *rows_per_s) {
    SF_ARG(rows_per_s, "rows_per_s is NULL");
    SF_ARG(n_rows >= 1 && n_rows <= (1ll << 31) - 2, "n_rows must be in [1, 2^31 - 2]");
    SF_ARG(row_bytes == 32 || row_bytes == 64 || row_bytes == 128 || row_bytes == 256,
           "row_bytes must be 32, 64, 128 or 256");
    SF_ARG(deg >= 4 && deg <= 256 && deg % 4 == 0, "deg must be a multiple of 4 in [4, 256]");
    SF_ARG(reps >= 1, "reps must be >= 1");
    cudaStream_t s = (cudaStream_t)stream;
    const int cols = row_bytes / 2;
    Scratch sc(s);
    uint16_t *T = nullptr;
    int32_t *idx = nullptr;
    float *out = nullptr;
    sf_status st;
    if ((st = sc.get(&T, (size_t)(n_rows + 1) * cols)) || (st = sc.get(&idx, (size_t)n_rows * deg)) ||
        (st = sc.get(&out, (size_t)n_rows * cols)))
        return st;
    const int fill_grid = 8 * sm_count();
    probe_fill_table<<<fill_grid, 256, 0, s>>>(T, n_rows + 1, cols);
    if ((st = check_launch("probe_fill_table"))) return st;
    probe_fill_idx<<<fill_grid, 256, 0, s>>>(idx, n_rows * deg, n_rows);
    if ((st = check_launch("probe_fill_idx"))) return st;
    const int grid = 4 * sm_count();
    auto launch = [&]() {
        switch (row_bytes) {
            case 32: probe_launch<2>(grid, s, T, idx, n_rows, deg, out, write_rows); break;
            case 64: probe_launch<4>(grid, s, T, idx, n_rows, deg, out, write_rows); break;
            case 128: probe_launch<8>(grid, s, T, idx, n_rows, deg, out, write_rows); break;
            default: probe_launch<16>(grid, s, T, idx, n_rows, deg, out, write_rows); break;
        }
        return check_launch("probe_gather_kernel");
    };
    for (int i = 0; i < 2; ++i)
        if ((st = launch())) return st;
    cudaEvent_t a = nullptr, b = nullptr;
    SF_CHECK_CUDA(cudaEventCreate(&a));
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return cuda_fail(cudaGetLastError(), "cudaEventCreate");
    }
    cudaEventRecord(a, s);
    for (int i = 0; i < reps && st == SF_OK; ++i) st = launch();
    cudaEventRecord(b, s);
    cudaError_t e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (st) return st;
    if (e != cudaSuccess) return cuda_fail(e, "timing the gather ceiling");
    *rows_per_s = (double)n_rows * deg * reps / ((double)ms * 1e-3);
    return SF_OK;
}

extern "C" SF_API sf_status sf_gather_ceiling(int64_t n_rows, int32_t row_bytes, int32_t deg, int32_t reps,
                                              void *stream, double *rows_per_s) {
    return gather_rate(n_rows, row_bytes, deg, reps, true, stream, rows_per_s);
}

extern "C" SF_API sf_status sf_gather_rate(int64_t n_rows, int32_t row_bytes, int32_t deg, int32_t reps,
                                           int32_t write_rows, void *stream, double *rows_per_s) {
    return gather_rate(n_rows, row_bytes, deg, reps, write_rows != 0, stream, rows_per_s);
}
