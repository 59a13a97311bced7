// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <vector>

#include "../../include/specfilt.h"

namespace sf {

// ---------------------------------------------------------------- errors
void set_error(const char *fmt, ...);
sf_status cuda_fail(cudaError_t e, const char *what);

#define SF_CHECK_CUDA(call)                                        \
    do {                                                           \
        cudaError_t _e = (call);                                   \
        if (_e != cudaSuccess) return ::sf::cuda_fail(_e, #call);  \
    } while (0)

#define SF_ARG(cond, ...)                 \
    do {                                  \
        if (!(cond)) {                    \
            ::sf::set_error(__VA_ARGS__); \
            return SF_ERR_ARG;            \
        }                                 \
    } while (0)

// Counts every kernel launch issued by the library; call after each launch.
void note_launch();
// Checks the launch that was just issued.
sf_status check_launch(const char *name);

// ---------------------------------------------------------------- memory
// Stream-ordered device allocation; zero bytes gives nullptr.
sf_status dev_alloc(void **p, size_t bytes, cudaStream_t s);
void dev_free(void *p, cudaStream_t s);

// RAII holder for stream-ordered allocations of one call.
struct Scratch {
    cudaStream_t s;
    std::vector<void *> ptrs;
    explicit Scratch(cudaStream_t st) : s(st) {}
    template <typename T>
    sf_status get(T **p, size_t count) {
        void *q = nullptr;
        sf_status st = dev_alloc(&q, count * sizeof(T), s);
        if (st != SF_OK) return st;
        if (q) ptrs.push_back(q);
        *p = static_cast<T *>(q);
        return SF_OK;
    }
    ~Scratch() {
        for (void *q : ptrs) dev_free(q, s);
    }
};

// ---------------------------------------------------------------- device info
int sm_count();
int current_device();

// ---------------------------------------------------------------- scans
// Exclusive prefix sum of n int32 values (out may alias in). The total must
// fit in int32. Uses stream-ordered temporaries.
sf_status exclusive_scan_i32(const int32_t *in, int32_t *out, int64_t n, cudaStream_t s);

// Deterministic sum of `count` doubles (fixed order), result in device *out.
sf_status reduce_sum_f64(const double *in, int64_t count, double *out, cudaStream_t s);

// ---------------------------------------------------------------- profiling
// Kernel variants are tagged mode * 3 + storage (SF_F32 0, SF_BF16 1,
// SF_F16 2) with mode 0 forward, 1 moments, 2 Clenshaw.
constexpr int kProfTags = 11;
constexpr int kProfTagAdjoint = 9;   // the adjoint's sampled-product kernel
constexpr int kProfTagKmeansTc = 10; // the k-means tensor-core distance kernel
bool profiling_on();
void profile_record(cudaEvent_t a, cudaEvent_t b, double bytes, int tag, int64_t launches = 1);
bool profile_events(cudaEvent_t *a, cudaEvent_t *b);
// A span times a run of consecutive launches of one kernel variant with one
// pair of events (per-launch events would add a bubble between launches);
// launches made while a span is open on this thread record no events.
bool profile_span_active();
void profile_span_set(bool on);
struct ProfSpan {
    cudaEvent_t a = nullptr, b = nullptr;
    cudaStream_t s = nullptr;
    bool on = false;
    int tag = 0;
    int64_t launches = 0;
    double bytes = 0.0;
    ProfSpan(cudaStream_t st, int t) : s(st), tag(t) {
        on = profiling_on() && !profile_span_active() && profile_events(&a, &b);
        if (on) {
            cudaEventRecord(a, s);
            profile_span_set(true);
        }
    }
    void add(double by) {
        ++launches;
        bytes += by;
    }
    ~ProfSpan() {
        if (!on) return;
        profile_span_set(false);
        cudaEventRecord(b, s);
        profile_record(a, b, bytes, tag, launches);
    }
};

// ---------------------------------------------------------------- host math
void cheb_coeffs_host(double lam_max, double lc, int p, int jackson, double *a);
double count_from_moments_host(const double *mu, int p, const double *a);
double tridiag_max_eig_host(int k, const double *a, const double *b);

}  // namespace sf

// Extra entries after rowptr[n] (holding nnz) and after colidx/val (zeros),
// so that 16-byte aligned bulk copies of any row or entry range stay inside
// the allocations.
constexpr int kCsrPad = 4;

// ---------------------------------------------------------------- objects
// Sliced-ELL copy of a CSR used by the sweep kernels (see sf_sell.cu).
namespace sf {
constexpr int kSliceRows = 8;  // rows per slice
}  // namespace sf
// The sweeps keep their signal blocks in slice-row order: block row t holds
// original row perm[t], so the rows of a tile are consecutive in memory, and
// `ridx` holds the column indices renumbered into that order. Rows t >= n are
// padding; row `rows` of every block is the zero row that padding entries
// gather.
struct SellMatrix {
    int32_t n = 0;
    int32_t n_slices = 0;
    int32_t rows = 0;         // n_slices * 8: a block has rows + 1 rows
    int64_t entries = 0;
    int32_t *sptr = nullptr;  // [n_slices + 1 + pad] entry offset of each slice
    int32_t *perm = nullptr;  // [n_slices * 8] original row of each slice row, -1 for none
    int32_t *idx = nullptr;   // [entries + pad] column index (original numbering), n for padding
    int32_t *ridx = nullptr;  // [entries + pad] column index as a slice row, `rows` for padding
    float *val = nullptr;     // [entries + pad] weight, 0 for padding; nullptr for unit weights
    int32_t *iperm = nullptr; // [n] slice row (slice * 8 + position) of each original row
    bool built = false;
};

namespace sf {
sf_status sell_build(SellMatrix *S, int32_t n, const int32_t *rowptr, const int32_t *colidx, const float *val,
                     cudaStream_t s);
void sell_release(SellMatrix *S);
// Stable LSD radix sort of 64-bit keys on bits [shift0, bits) (8 bits per
// pass), carrying `vals` when non-null; keys/vals end up in the returned
// pointers (the _alt buffers are the ping-pong partners).
sf_status radix_sort(uint64_t *&keys, float *&vals, uint64_t *&keys_alt, float *&vals_alt, int64_t count,
                     int shift0, int bits, cudaStream_t s);
}  // namespace sf

struct sf_graph {
    int32_t n = 0;
    int64_t nnz = 0;  // stored off-diagonal entries
    int32_t *rowptr = nullptr;
    int32_t *colidx = nullptr;
    float *val = nullptr;
    double *strength = nullptr;
    double max_strength = 0.0;
    int32_t unit_weights = 1;
    int32_t normalized = 0;  // the diagonal (strength) is 1 / 0, not the row sums: I - S^-1/2 W S^-1/2
    int device = 0;
    mutable SellMatrix sell;
    mutable std::mutex sell_mu;
};

struct sf_batch {
    int32_t n_graphs = 0;
    int32_t n = 0;
    int64_t nnz = 0;
    int32_t *rowptr = nullptr;
    int32_t *colidx = nullptr;
    float *val = nullptr;
    double *strength = nullptr;
    int32_t *row_graph = nullptr;  // graph id of each row
    int32_t unit_weights = 1;
    std::vector<int32_t> offsets;   // host, n_graphs + 1
    std::vector<int64_t> nnz_offsets;
    int device = 0;
    mutable SellMatrix sell;
    mutable std::mutex sell_mu;
};

// Strength recomputation (shared by build and set_values).
namespace sf {
sf_status compute_strength(sf_graph *g, cudaStream_t s);
}
