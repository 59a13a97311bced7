/*
 * specfilt.h -- C ABI of the GB300 graph-filtering library (libspecfilt.so).
 *
 * The library computes the hot path of accelerated spectral clustering by
 * graph filtering of random signals (Tremblay, Puy, Borgnat, Gribonval,
 * Vandergheynst): a polynomial approximation of the ideal low-pass filter of
 * Eq. (2) applied by repeated sparse products with the Laplacian L = S - W
 * (§2.1, §2.4 Eq. (3)) to a block R of random signals (§3.1), the
 * eigenvalue count and dichotomy built on it (§3.2), the largest-eigenvalue
 * estimate it needs (§4.1 step 1) and the feature rows it yields (Eq. (6),
 * Eq. (11)). The polynomial is expanded in the Chebyshev basis of
 * Lt = (2 / lam_max) L - I, so every filter order is one sparse-times-dense
 * product T_j = 2 Lt T_{j-1} - T_{j-2}.
 *
 * Conventions shared by every entry point:
 *   - Return value: SF_OK (0) or an error status; nothing is thrown.
 *     sf_last_error() gives a message for the calling thread's last failure.
 *   - Pointers documented "device" are CUDA device (or managed) memory on
 *     the current device; "host" pointers are ordinary CPU memory.
 *   - Ownership: the caller owns every buffer it passes. Objects the library
 *     creates (sf_graph, sf_batch) are freed with their *_free function.
 *     Internal work buffers are stream-ordered allocations released before
 *     the call returns or at the end of its stream work.
 *   - Streams: `stream` is a cudaStream_t (NULL = legacy default stream).
 *     Calls are asynchronous on that stream unless they return host values,
 *     in which case they synchronise it before returning (stated per call).
 *   - Layouts: signal blocks are row-major N x n_sig (one row per node,
 *     signals contiguous); coefficient tables are row-major
 *     [n_cut][p + 1]; graphs are CSR with int32 indices and fp32 weights.
 *   - Errors from bad arguments leave outputs untouched. A CUDA failure
 *     returns SF_ERR_CUDA and leaves outputs undefined.
 */
#ifndef SPECFILT_H
#define SPECFILT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define SF_API __attribute__((visibility("default")))
#else
#define SF_API
#endif

/* Status codes. */
enum {
    SF_OK = 0,
    SF_ERR_ARG = 1,      /* invalid argument (sizes, pointers, graph content) */
    SF_ERR_CUDA = 2,     /* a CUDA runtime call or kernel failed */
    SF_ERR_OOM = 3,      /* device allocation failed */
    SF_ERR_TIMEOUT = 4,  /* a bounded device wait gave up */
    SF_ERR_NUMERIC = 5   /* non-finite value detected where a finite one is required */
};
typedef int32_t sf_status;

/* Element types of signal blocks. */
enum { SF_F32 = 0, SF_BF16 = 1, SF_F16 = 2 };

/* Filter algorithms. */
enum {
    SF_ALGO_AUTO = 0,     /* Clenshaw for one cutoff with FP32 blocks, else the forward recurrence */
    SF_ALGO_FORWARD = 1,  /* T_j blocks forward, Y_c += a_cj T_j for every cutoff c */
    SF_ALGO_CLENSHAW = 2  /* backward Clenshaw sum, one cutoff at a time */
};

/*
 * Memory-system hints of the sweep kernels (sf_opts.sweep_hints: 0 = the
 * library default, SF_HINT_IDX_EVICT_FIRST | SF_HINT_OUT_STREAMING |
 * SF_HINT_MIXED_ADD; SF_HINTS_NONE; or any OR of these). They change where
 * data is cached or how a sum is issued, never the value of a result.
 */
enum {
    SF_HINTS_NONE = -1,
    SF_HINT_IDX_EVICT_FIRST = 1, /* staged index copies read with an L2 evict-first policy */
    SF_HINT_OUT_STREAMING = 2,   /* T_j / b_j stores marked streaming (evict-first) */
    SF_HINT_MIXED_ADD = 8        /* unit weights, 16-bit blocks: FP32 += 16-bit adds in one instruction */
};

/* Sweep kernel variants (sf_opts.sweep_kernel). */
enum {
    SF_SWEEP_AUTO = 0,   /* the staged tiles (SF_SWEEP_TILED) unless sf_autotune chose otherwise */
    SF_SWEEP_TILED = 1,  /* CTA tiles whose indices are staged in shared memory by TMA bulk copies */
    SF_SWEEP_DIRECT = 2, /* no staging: each warp reads its rows' indices from global memory */
    SF_SWEEP_PERSISTENT = 3 /* batches: one persistent launch runs every order (per-graph arrival
                               counters); single graphs and the moment sweep use the staged tiles */
};

/*
 * Tuning and precision options; a NULL sf_opts* means all zero (defaults).
 *   storage         SF_F32 / SF_BF16 / SF_F16: element type of the T_j (or
 *                   Clenshaw b_j) blocks kept between orders. Products and
 *                   accumulations are FP32 in every case; the output Y is FP32.
 *                   With SF_F16 each column slab of R is first scaled by the
 *                   power of two that puts its largest magnitude in (1/2, 1]
 *                   (exact, undone on output), which keeps the blocks inside
 *                   the FP16 range. The moment sweep rejects SF_F16.
 *   algo            SF_ALGO_*.
 *   slab_cols       signal columns processed per sweep (0 = automatic: the
 *                   widest power-of-two slab whose gathered block fits in
 *                   64 MB, about half of L2, and at least 16 FP32 or 32
 *                   16-bit columns). The signals are independent, so the
 *                   block is filtered in column slabs.
 *   block_warps     warps per thread block of the sweep kernel (0 = automatic).
 *   blocks_per_sm   resident blocks per SM of the persistent sweep grid (0 = max).
 *   ckpt_every      adjoint only: 0 = automatic (store every T_j when it fits
 *                   under mem_cap_mb, else checkpoint), 1 = store all, k > 1 =
 *                   keep every k-th pair of blocks and recompute the rest.
 *   mem_cap_mb      adjoint only: memory budget for stored T_j blocks (0 = 16384).
 *   carveout_pct    shared-memory share of the L1/shared array requested for
 *                   the sweep kernel, in percent (0 = driver default). The L1
 *                   share holds the gathers in flight, so large values slow
 *                   the sweep down.
 *   l2_window       1: mark each order's gathered block as persisting in L2
 *                   (access-policy window, up to the device's persisting
 *                   set-aside, which the call raises to its maximum); 0: no
 *                   window. At the end of such a call the stream is
 *                   synchronised, the persisting lines are turned back to
 *                   normal and the set-aside is put back to its previous size
 *                   (not while the stream is being captured). Measured slower
 *                   than no window on the 1M-node workload; sf_autotune does
 *                   not select it.
 *   sweep_kernel    SF_SWEEP_*: which sweep kernel runs the orders. Both sum
 *                   each row in the same order, so blocks and filter outputs
 *                   are bit-identical; the FP64 moment sums may differ in the
 *                   last bits (rows reach the block partial sums in another
 *                   order).
 *   sweep_hints     SF_HINT_* mask, SF_HINTS_NONE, or 0 for the default.
 */
typedef struct sf_opts {
    int32_t storage;
    int32_t algo;
    int32_t slab_cols;
    int32_t block_warps;
    int32_t blocks_per_sm;
    int32_t ckpt_every;
    int64_t mem_cap_mb;
    int32_t carveout_pct;
    int32_t l2_window;
    int32_t sweep_kernel;
    int32_t sweep_hints;
} sf_opts;

typedef struct sf_graph sf_graph; /* device-resident CSR of W, owned by the library */
typedef struct sf_batch sf_batch; /* block-diagonal concatenation of several graphs */

/* ---------------------------------------------------------------------- */
/* Status helpers                                                          */
/* ---------------------------------------------------------------------- */

/* Static text for a status code. */
SF_API const char *sf_status_str(sf_status s);
/* Message describing the calling thread's most recent failure ("" if none). */
SF_API const char *sf_last_error(void);
/* ABI version (major * 100 + minor). */
SF_API int32_t sf_version(void);
/* Number of CUDA kernels this library has launched in this process. */
SF_API int64_t sf_launch_count(void);

/* ---------------------------------------------------------------------- */
/* Graph construction (§2: W_ij = W_ji >= 0; §2.1: s_i = sum_{j != i} W_ij) */
/* ---------------------------------------------------------------------- */

/*
 * Build the symmetric CSR of W from an undirected edge list.
 *   n_nodes   number of nodes N (>= 1)
 *   n_edges   number of listed edges m (>= 0); 2 m must be < 2^31
 *   src, dst  device int32[m], endpoints in [0, N)
 *   w         device float[m], weights (finite, >= 0), or NULL for all 1
 * Each edge (u, v, w) with u != v yields W_uv and W_vu; self-loops are
 * dropped (the strength of §2.1 excludes j = i); repeated pairs keep the
 * largest weight. Columns are sorted within each row, so the result is
 * bit-identical for any order of the edge list. Also computes the strengths
 * s_i (FP64) and whether every stored weight equals 1.
 * Synchronises `stream` (the entry count must be known). Errors: SF_ERR_ARG
 * for an endpoint out of range or a negative / non-finite weight.
 */
SF_API sf_status sf_csr_build(int32_t n_nodes, int64_t n_edges, const int32_t *src, const int32_t *dst,
                              const float *w, void *stream, sf_graph **out);

/* Sizes: N, stored off-diagonal entries, and 1 when every weight is 1. Host outputs, any may be NULL. */
SF_API sf_status sf_graph_info(const sf_graph *g, int32_t *n, int64_t *nnz_off, int32_t *unit_weights,
                               double *max_strength);

/* Borrowed device views of the CSR (valid until sf_graph_free); any may be NULL. */
SF_API sf_status sf_graph_csr(const sf_graph *g, const int32_t **rowptr, const int32_t **colidx,
                              const float **val, const double **strength);

/*
 * Replace the stored weights (same pattern) and recompute strengths.
 *   val  device float[nnz_off] in CSR order; must be symmetric (W_uv = W_vu)
 *        and >= 0 -- the symmetry is the caller's contract, not checked.
 * Synchronises `stream` (the largest strength is read back).
 */
SF_API sf_status sf_graph_set_values(sf_graph *g, const float *val, void *stream);

/*
 * The normalised Laplacian I - S^{-1/2} W S^{-1/2} (the footnote of §2.1,
 * "other types of Laplacians, such as the normalized Laplacian") as a new
 * graph: weights w_ij / sqrt(s_i s_j) (FP64, rounded to FP32) and an explicit
 * diagonal 1 in place of the row sums (0 for an isolated node). Every
 * filtering entry point then works on it unchanged (its spectrum lies in
 * [0, 2], so sf_lambda_max_estimate's bound is 2); sf_graph_set_values and
 * sf_cheb_filter_backward reject it. The caller frees *out with
 * sf_graph_free. Synchronises `stream`.
 */
SF_API sf_status sf_graph_normalize(const sf_graph *g, void *stream, sf_graph **out);

SF_API void sf_graph_free(sf_graph *g);

/* ---------------------------------------------------------------------- */
/* The order m* (§2.4, criterion (4))                                      */
/* ---------------------------------------------------------------------- */

/*
 * The smallest order m in [1, p_max] whose Chebyshev approximation (Jackson-
 * damped when `jackson`) of the ideal low-pass h_x on [0, 1] (h = 1 for
 * t <= x) stays within delta of h at every point t of the grid g / 4095
 * (g = 0..4095) and the band edges x +- w with |t - x| >= w; *m_star = -1 when
 * no order up to p_max does. x = lambda_c / lambda_N. The criterion of §2.4
 * takes the sup over all of [0, lambda_N], which no polynomial can bring
 * below 1/2 at the jump: the band of half-width w (a fraction of lambda_N)
 * around it is left out. Host only; the paper's tolerance is delta = 0.1.
 */
SF_API sf_status sf_cheb_order(double x, double delta, double w, int32_t jackson, int32_t p_max, int32_t *m_star);

/* ---------------------------------------------------------------------- */
/* lambda_N (§4.1 step 1)                                                  */
/* ---------------------------------------------------------------------- */

/*
 * Largest Laplacian eigenvalue estimate by `iters` Lanczos steps in FP64 on
 * the device (no re-orthogonalisation; the largest Ritz value is unaffected
 * by the loss of orthogonality), the tridiagonal solved on the host.
 *   v0        device double[N] start vector, or NULL to draw one from the
 *             SplitMix64 sequence seeded by `seed` (uniform in [-1, 1))
 *   theta_max host out: largest Ritz value (<= lambda_N)
 *   lam_hat   host out: min(1.01 * theta_max, 2 * max_i s_i), the value the
 *             filters should use (1 for an edgeless graph)
 * Synchronises `stream`.
 */
SF_API sf_status sf_lambda_max_estimate(const sf_graph *g, int32_t iters, const double *v0, uint64_t seed,
                                        void *stream, double *theta_max, double *lam_hat);

/* ---------------------------------------------------------------------- */
/* Coefficients of the ideal low-pass Eq. (2) (host, FP64)                 */
/* ---------------------------------------------------------------------- */

/*
 * Chebyshev coefficients of h_lc on [0, lam_max] for each cutoff:
 * coeffs[c][0] = 1 - theta_c / pi, coeffs[c][j] = -2 sin(j theta_c) / (pi j),
 * theta_c = arccos(clamp(2 lc / lam_max - 1, -1, 1)); with jackson != 0 each
 * term is multiplied by the Jackson factor g_j of a degree-p expansion.
 *   cutoffs host double[n_cut]; coeffs host double[n_cut][p + 1].
 */
SF_API sf_status sf_cheb_coeffs(double lam_max, const double *cutoffs, int32_t n_cut, int32_t p,
                                int32_t jackson, double *coeffs);

/* ---------------------------------------------------------------------- */
/* Fast filtering of random signals (§2.4 Eq. (3), §3.1 Eq. (6), §4.1 step 5) */
/* ---------------------------------------------------------------------- */

/*
 * Y_c = sum_{j=0}^{p} coeffs[c][j] T_j(Lt) R for c = 0..n_cut-1.
 *   lam_max  the lam_hat used for Lt (> 0)
 *   coeffs   host double[n_cut][p + 1] (p >= 0, 1 <= n_cut <= 64)
 *   R        device N x n_sig block, element type r_dtype (SF_F32 or SF_BF16)
 *   Y        device float[n_cut][N][n_sig]
 * Asynchronous on `stream`.
 */
SF_API sf_status sf_cheb_filter(const sf_graph *g, double lam_max, const double *coeffs, int32_t n_cut,
                                int32_t p, const void *R, int32_t r_dtype, int32_t n_sig, float *Y,
                                const sf_opts *opts, void *stream);

/*
 * Chebyshev moments mu_m = <R, T_m(Lt) R>_F, m = 0..2p, from one sweep of p
 * orders: mu_{2j} = 2 <T_j R, T_j R> - mu_0 and
 * mu_{2j-1} = 2 <T_j R, T_{j-1} R> - mu_1 (products of Chebyshev
 * polynomials). Per-row partial sums in FP32, everything across rows in
 * FP64 with a fixed reduction order (deterministic).
 *   moments host double[2p + 1]. Synchronises `stream`.
 * SF_ERR_NUMERIC when a moment is not finite or ||T_j R||^2 exceeds
 * 16 ||R||^2 (lam_max below the largest Laplacian eigenvalue: the recurrence
 * diverges for eigenvalues beyond it).
 */
SF_API sf_status sf_cheb_moments(const sf_graph *g, double lam_max, const void *R, int32_t r_dtype,
                                 int32_t n_sig, int32_t p, double *moments, const sf_opts *opts,
                                 void *stream);

/*
 * Eigenvalue count of §3.2 from moments (host, FP64):
 * counts[c] = sum_{j,j'} a_cj a_cj' (mu_{j+j'} + mu_{|j-j'|}) / 2, i.e. the
 * squared Frobenius norm of the filtered block. moments: host double[2p + 1].
 */
SF_API sf_status sf_count_from_moments(const double *moments, int32_t p, const double *coeffs,
                                       int32_t n_cut, double *counts);

/*
 * sf_cheb_moments followed by coefficients (with or without Jackson
 * damping) and counts for every cutoff. counts: host double[n_cut];
 * moments_out: host double[2p + 1] or NULL. Synchronises `stream`.
 */
SF_API sf_status sf_eigencount(const sf_graph *g, double lam_max, const void *R, int32_t r_dtype,
                               int32_t n_sig, int32_t p, const double *cutoffs, int32_t n_cut,
                               int32_t jackson, double *counts, double *moments_out, const sf_opts *opts,
                               void *stream);

/*
 * Dichotomy of §3.2 on [0, lam_max] (host, FP64, on moments -- no GPU work):
 * the smallest cutoff whose count reaches k, by bisection stopped after
 * max_iter halvings or when the bracket is below tol * lam_max; returns the
 * bracket's upper end in *lam_k.
 */
SF_API sf_status sf_dichotomy(const double *moments, int32_t p, double lam_max, double k, int32_t jackson,
                              int32_t max_iter, double tol, double *lam_k);

/*
 * Feature rows f~_i (Eq. (6), Eq. (11)): F = Y, or with normalize != 0 each
 * row divided by its Euclidean norm (norm in FP64; all-zero rows stay zero).
 *   Y, F  device float[N][n_sig] (F may alias Y). Asynchronous.
 */
SF_API sf_status sf_features(const float *Y, int32_t n, int32_t n_sig, int32_t normalize, float *F,
                             void *stream);

/*
 * Feature normalisation when the signal columns are spread over several
 * devices (each holds a column shard of Y): every device computes its rows'
 * partial sums of squares, the caller adds them across devices (one
 * all-reduce of N doubles), then every device scales its shard by the total.
 *   sf_row_sumsq:       sumsq[i] = sum_c Y[i][c]^2 (device double[N]; FP32
 *                       per-lane partials combined in FP64)
 *   sf_features_scaled: F[i][c] = Y[i][c] / sqrt(sumsq[i]), zero rows stay
 *                       zero (F may alias Y)
 * With the full Y on one device the two calls equal sf_features(..., 1, ...).
 * Asynchronous.
 */
SF_API sf_status sf_row_sumsq(const float *Y, int32_t n, int32_t n_sig, double *sumsq, void *stream);
SF_API sf_status sf_features_scaled(const float *Y, int32_t n, int32_t n_sig, const double *sumsq, float *F,
                                    void *stream);

/* ---------------------------------------------------------------------- */
/* Adjoint (reverse mode) of the filter                                    */
/* ---------------------------------------------------------------------- */

/*
 * Gradients of l = <G, Y>_F for Y = sum_j coeffs[j] T_j(Lt) R (one cutoff),
 * lam_max held fixed:
 *   grad_val     device float[nnz_off]: dl/dW_uv for the undirected edge of
 *                each stored entry (both directions carry the same value),
 *                = (2 / lam_max)(M_uu + M_vv - M_uv - M_vu), with
 *                M = Gb_1 T_0^T + sum_{j>=2} 2 Gb_j T_{j-1}^T on the pattern
 *   grad_coeffs  host double[p + 1]: <G, T_j R>  (may be NULL)
 *   grad_R       device float[N][n_sig]: sum_j coeffs[j] T_j(Lt) G (may be NULL)
 * Gb_j run the Clenshaw recurrence on G top-down (Lt is symmetric). T_j
 * blocks are stored or recomputed from checkpoints per opts (ckpt_every,
 * mem_cap_mb). G and R are FP32. Synchronises `stream` when grad_coeffs
 * is non-NULL.
 */
SF_API sf_status sf_cheb_filter_backward(const sf_graph *g, double lam_max, const double *coeffs, int32_t p,
                                         const float *R, int32_t n_sig, const float *G, float *grad_val,
                                         double *grad_coeffs, float *grad_R, const sf_opts *opts,
                                         void *stream);

/* ---------------------------------------------------------------------- */
/* Many graphs in one sweep                                                */
/* ---------------------------------------------------------------------- */

/*
 * Concatenate graphs into one block-diagonal CSR (node ids offset by the
 * preceding graphs' sizes). The source graphs may be freed afterwards.
 * Synchronises `stream`.
 */
SF_API sf_status sf_batch_build(const sf_graph *const *graphs, int32_t n_graphs, void *stream,
                                sf_batch **out);

/* Total nodes, total stored entries, number of graphs; row offsets host int32[n_graphs + 1] (may be NULL). */
SF_API sf_status sf_batch_info(const sf_batch *b, int32_t *n_total, int64_t *nnz_total, int32_t *n_graphs,
                               int32_t *row_offsets);

SF_API void sf_batch_free(sf_batch *b);

/*
 * Filter every graph of the batch with its own lam_max and coefficients
 * (the fast filtering of §2.4 on each graph). With opts->sweep_kernel =
 * SF_SWEEP_PERSISTENT one kernel launch runs all p orders of a column slab:
 * blocks take (order, tile) items from a queue, and a tile starts an order as
 * soon as every graph its rows belong to has finished the previous order on
 * all of its tiles (per-graph arrival counters), so small graphs do not wait
 * for the batch's largest graph at every order. Every such wait is bounded:
 * one that runs out sets the device status word (sf_device_check then returns
 * SF_ERR_TIMEOUT) and makes the launch's other waits give up. Otherwise
 * (SF_SWEEP_AUTO, SF_SWEEP_TILED, SF_SWEEP_DIRECT) one launch per order
 * covers all graphs. Both forms compute every row with the same operations:
 * their outputs are bit-identical.
 *   lam_max  host double[n_graphs]
 *   coeffs   host double[n_graphs][p + 1]
 *   R, Y     device blocks of sum(N_g) rows x n_sig, graph g's rows at its
 *            row offset; R of type r_dtype, Y float.
 * Asynchronous on `stream`.
 */
SF_API sf_status sf_cheb_filter_batched(const sf_batch *b, const double *lam_max, const double *coeffs,
                                        int32_t p, const void *R, int32_t r_dtype, int32_t n_sig, float *Y,
                                        const sf_opts *opts, void *stream);

/*
 * sf_cheb_filter_batched with n_cut coefficient rows per graph (several
 * cutoffs lambda_c per graph, accumulated in one forward sweep; Clenshaw,
 * when asked for, runs one cutoff at a time).
 *   coeffs   host double[n_graphs][n_cut][p + 1], 1 <= n_cut <= 64
 *   Y        device float[n_cut][sum(N_g)][n_sig]
 * Asynchronous on `stream`.
 */
SF_API sf_status sf_cheb_filter_batched_multi(const sf_batch *b, const double *lam_max, const double *coeffs,
                                              int32_t n_cut, int32_t p, const void *R, int32_t r_dtype,
                                              int32_t n_sig, float *Y, const sf_opts *opts, void *stream);

/*
 * sf_cheb_moments without any device allocation. The paper has no
 * counterpart: this entry point exists for callers that cannot allocate
 * device memory when they need the moments -- frameworks whose own caching
 * allocator owns all device memory and forbids foreign allocations, and
 * latency-bound loops that cannot afford an allocator call (cudaFree
 * synchronises the device). Its working memory is one fixed 64 MiB array in
 * the library's device image, held by every GPU that loads the library until
 * the process exits.
 *   R        device float[N][n_sig] (FP32 signals; blocks are FP32)
 *   moments  host double[2p + 1]: the moments of sf_cheb_moments, equal to
 *            that entry point's within the FP64 reduction-order tolerance
 *            (the two may cut the block into different column slabs)
 * Requirements and behaviour:
 *   - the graph must already have its sweep layout, which the first
 *     sf_cheb_moments / sf_cheb_filter / sf_autotune call on it builds
 *     (SF_ERR_ARG otherwise);
 *   - the column slab halves (down to 8 columns) until three FP32 blocks of
 *     the graph and the small tables fit the array; SF_ERR_ARG beyond that,
 *     about 670,000 rows for moderate p (the limit does not depend on n_sig);
 *   - the same finiteness and growth checks as sf_cheb_moments
 *     (SF_ERR_NUMERIC for non-finite signals or lam_max below the spectrum);
 *   - the first call on a device looks up the array's address; make that
 *     call before any stream capture;
 *   - calls share the array: calls whose GPU work can overlap (unordered
 *     streams) race; each call clears what must start at zero;
 *   - no cudaMalloc, cudaFree or allocating library routine is called.
 * Synchronises `stream`.
 */
SF_API sf_status sf_cheb_moments_noalloc(const sf_graph *g, double lam_max, const float *R, int32_t n_sig,
                                         int32_t p, double *moments, void *stream);

/*
 * Synchronise `stream` and report whether a sweep kernel gave up a bounded
 * wait for its staged CSR tile since the last check (SF_ERR_TIMEOUT; the
 * flag is then cleared). Entry points that synchronise check it themselves;
 * asynchronous ones (sf_cheb_filter, sf_cheb_filter_batched) leave it to
 * this call.
 */
SF_API sf_status sf_device_check(void *stream);

/*
 * sf_cheb_filter_batched with its tables already on the device, for capture
 * into a CUDA graph: the call copies nothing between host and device and
 * never synchronises (work buffers are stream-ordered allocations, which a
 * graph captures as allocation nodes).
 *   two_over_lam  device double[n_graphs]: 2 / lam_max of each graph
 *   coeffs        device float[n_graphs][p + 1]
 * The batch's sweep layout must exist (a first sf_cheb_filter_batched call
 * builds it; SF_ERR_ARG otherwise), and so must the L2 set-up when
 * opts->l2_window is 1 (done by the first call with a window).
 */
SF_API sf_status sf_cheb_filter_batched_dev(const sf_batch *b, const double *two_over_lam, const float *coeffs,
                                            int32_t p, const void *R, int32_t r_dtype, int32_t n_sig, float *Y,
                                            const sf_opts *opts, void *stream);

/* ---------------------------------------------------------------------- */
/* Tile autotuner and kernel timing                                        */
/* ---------------------------------------------------------------------- */

/*
 * Time candidate tile shapes (slab width, warps per block, shared carveout,
 * L2 window) of the sweep kernel on this graph for n_sig signals and the given storage
 * type, a few orders each, and write the fastest into *best (other fields
 * copied from *base, which may be NULL). Candidates are ranked by the summed
 * duration of their sweep-kernel launches (the kernel timing hooks below,
 * which this call uses and leaves off). Results are cached per
 * (N, nnz, n_sig, storage, n_cut, device) in the process. Synchronises
 * `stream`.
 */
SF_API sf_status sf_autotune(const sf_graph *g, int32_t n_sig, int32_t storage, int32_t n_cut,
                             const sf_opts *base, void *stream, sf_opts *best);

/*
 * Kernel timing of the sweep kernel: after sf_profile_begin(), every launch
 * of the per-order sweep kernel is bracketed by CUDA events on its stream.
 * sf_profile_end() synchronises those events and returns the number of
 * timed launches, their summed duration (ms) and their summed algorithmic
 * bytes (compulsory traffic: CSR once, gathered rows once, streamed blocks).
 */
SF_API sf_status sf_profile_begin(void);
SF_API sf_status sf_profile_end(int64_t *launches, double *ms, double *bytes);
/*
 * Per-variant totals of the last sf_profile_end: tag = 3 * mode + storage,
 * with mode 0 forward, 1 moments, 2 Clenshaw and storage SF_F32 / SF_BF16 /
 * SF_F16; tag 9 is the adjoint kernel of sf_cheb_filter_backward, tag 10
 * the tensor-core distance kernel of sf_kmeans.
 */
SF_API sf_status sf_profile_variant(int32_t tag, int64_t *launches, double *ms, double *bytes);

/* ---------------------------------------------------------------------- */
/* k-means on the feature rows (§4.1 step 6)                               */
/* ---------------------------------------------------------------------- */

enum {
    SF_KMEANS_AUTO = 0,         /* tensor cores when the shape allows (below), else CUDA cores */
    SF_KMEANS_TENSOR = 1,       /* tensor cores (SF_ERR_ARG when the shape does not allow them) */
    SF_KMEANS_CUDA_CORES = 2,   /* CUDA cores only */
    SF_KMEANS_TENSOR_SINGLE = 3 /* tensor cores, one TF32 product per pair (no split operands) */
};

/*
 * Lloyd's k-means with the Euclidean distance between feature rows (§4.1
 * step 6), from given initial centroids.
 *   F         device float[n][d], row-major, rows f~_i (e.g. sf_features output)
 *   n, d, k   rows (>= 1), columns (1..4096), clusters (1..1023)
 *   C         device float[k][d]: initial centroids in, final centroids out
 *   max_iter  maximum number of assignments (>= 1)
 *   mode      SF_KMEANS_*
 *   labels    device int32[n] out: cluster of each row
 *   iters     host out: assignments performed
 *   inertia   host out or NULL: sum over rows (FP64) of the squared distance
 *             to the centroid of the last assignment
 * Iteration: assignment label_i = argmin_c d(f_i, c_c), ties to the lowest c,
 * with d the FP32 fused-multiply-add sum of (f_ij - c_cj)^2 in index order;
 * stop when no label changed (from the second assignment on); otherwise
 * c_c = (sum of its rows / count) rounded to FP32, empty clusters keeping
 * their centroid, the sum exact over the values rounded down to multiples
 * of 2^-sh, with n max|F_ij| 2^sh just below 2^62. With tensor cores (d a
 * multiple of 32 in [32, 128], k <= 128, F and C 16-byte aligned) the
 * products f_i.c_c come from tcgen05 TF32 MMAs: with F and C split into TF32
 * high and low parts (three MMAs per product; 8 n d bytes of device memory
 * more) for SF_KMEANS_AUTO and SF_KMEANS_TENSOR, one product per pair for
 * SF_KMEANS_TENSOR_SINGLE. Every row whose two best candidates lie within
 * the products' error bound is decided again with the exact FP32 sum on
 * CUDA cores, so all modes return the same labels. Deterministic.
 * SF_ERR_NUMERIC when a row or a centroid is not finite (labels and C are
 * then unspecified). The host reads whether an assignment changed labels
 * one assignment later, while the GPU runs on (an update after the final
 * assignment leaves C as it was); synchronises `stream` before returning.
 */
SF_API sf_status sf_kmeans(const float *F, int32_t n, int32_t d, int32_t k, float *C, int32_t max_iter,
                           int32_t mode, int32_t *labels, int32_t *iters, double *inertia, void *stream);

/* ---------------------------------------------------------------------- */
/* Stability of the clusterings (§4.3, Eq. (12))                           */
/* ---------------------------------------------------------------------- */

/*
 * Adjusted Rand index (Hubert and Arabie 1985) of two labelings, the
 * similarity §4.3 averages in Eq. (12).
 *   a, b    device int32[n], labels in [0, ka) and [0, kb) (SF_ERR_ARG otherwise)
 *   ka, kb  label ranges, ka * kb <= 2^24
 *   ari     host out
 * Contingency counts on the device (integer atomics: deterministic), the
 * formula in FP64 on the host. Synchronises `stream`.
 */
SF_API sf_status sf_adjusted_rand(const int32_t *a, const int32_t *b, int32_t n, int32_t ka, int32_t kb,
                                  void *stream, double *ari);

/*
 * gamma(k) of §4.3, Eq. (12), for k = kmin..kmax: the mean adjusted Rand
 * index between the clusterings of J realisations of the eta random signals.
 *   p           order of the count's moment sweep
 *   p_filter    order of the filters: > 0 as given (<= 20000); 0 picks the
 *               order at which the filters of adjacent k differ: in
 *               theta = arccos(2 lambda / lam_max - 1) a Jackson-damped series
 *               of order q has a transition of standard deviation about
 *               pi / (q + 2), and the order makes +-2 of them fit in the
 *               smallest theta gap between the cutoffs of k - 1 .. kmax + 1
 *               (q + 2 >= 4 pi / gap, at least p, at most 20000). The cutoffs
 *               always come from the count at order p.
 *   Rc          device float[N][eta]: the count's probe block; lam_k is the
 *               dichotomy of the moments for the count k - 1/2 (one moment
 *               sweep serves every k)
 *   R           device float[J][N][eta]: the J realisations, filtered side by
 *               side as one block of J * eta columns at every lam_k in one
 *               forward sweep (Jackson damping); each realisation's rows are
 *               normalised and clustered by sf_kmeans into k clusters from
 *               `starts` seeded starts (lowest inertia kept)
 *   max_iter    k-means assignments per start
 *   seed        start rows: SplitMix64 (Steele, Lea, Flood 2014) of
 *               (j << 40) | (k << 20) | (t << 10) | c, modulo N, for start t
 *               of realisation j, centroid c
 *   opts        block storage and tiles of the sweeps (the algorithm is forward)
 *   gamma       host out double[kmax - kmin + 1]; lam_k host out, same length
 *   p_used      host out: the filter order used (NULL: not reported)
 * Needs J >= 2, J * eta <= 2^20, 1 <= kmin <= kmax <= 1023, starts <= 1023.
 * Synchronises `stream`.
 */
SF_API sf_status sf_stability(const sf_graph *g, double lam_max, int32_t p, int32_t p_filter, const float *Rc,
                              const float *R, int32_t J, int32_t eta, int32_t kmin, int32_t kmax, int32_t max_iter,
                              int32_t starts, uint64_t seed, const sf_opts *opts, void *stream, double *gamma,
                              double *lam_k, int32_t *p_used);

/*
 * Self-test of the failure path (no counterpart in the paper): one block
 * waits on an mbarrier that nothing completes, gives up after `polls` polls
 * (1..2^20) and sets the device status word exactly as a sweep kernel whose
 * staged copy never landed would; the next sf_device_check then returns
 * SF_ERR_TIMEOUT and clears the word. Nothing faults and the context stays
 * usable. Asynchronous on `stream`.
 */
SF_API sf_status sf_selftest_bounded_wait(int32_t polls, void *stream);

/*
 * Self-test of the persistent batch sweep's failure path (no counterpart in
 * the paper): one thread waits, with the batch kernel's own wait, for a graph
 * whose arrival counter nothing increments, gives up after `polls` polls
 * (1..2^16, 128 ns apart) and sets the device status word and the launch's
 * abort flag as the batch kernel does; the next sf_device_check returns
 * SF_ERR_TIMEOUT and clears the word. Nothing faults. Synchronises `stream`.
 */
SF_API sf_status sf_selftest_arrival_wait(int32_t polls, void *stream);

/*
 * Measured ceiling of the sweep's gather pattern. A diagnostic with no
 * counterpart in the paper: it times a kernel that does nothing but the
 * sweep's data movement without its arithmetic -- for every output row, sum
 * (in FP32) `deg` uniformly random rows of a synthetic BF16 table of
 * n_rows + 1 rows of row_bytes bytes, with lane groups of row_bytes / 16
 * lanes, eight 16-byte gathers in flight per lane, indices read from memory,
 * FP32 sums written out -- so a sweep launch's duration can be set against
 * what the memory system delivers for the same random-row pattern.
 *   n_rows      table rows and output rows (1 .. 2^31 - 2)
 *   row_bytes   32, 64, 128 or 256
 *   deg         entries per output row: a multiple of 4 in [4, 256]
 *   reps        timed launches (>= 1) after two untimed ones
 *   rows_per_s  out: gathered rows per second (mean over the timed launches)
 * Allocates and frees its own buffers: (n_rows + 1) * row_bytes (table),
 * n_rows * deg * 4 (indices), n_rows * row_bytes * 2 (sums). Synchronises
 * `stream`.
 */
SF_API sf_status sf_gather_ceiling(int64_t n_rows, int32_t row_bytes, int32_t deg, int32_t reps, void *stream,
                                   double *rows_per_s);

/*
 * sf_gather_ceiling with the write-back made optional (a diagnostic with no
 * counterpart in the paper). write_rows != 0 is sf_gather_ceiling itself;
 * write_rows == 0 writes one float per output row instead of the row's sums,
 * so the timing is that of the random-row gathers (and their index reads)
 * alone: the rate the memory system sustains for the pattern with nothing
 * else in flight. Arguments, buffers and errors as for sf_gather_ceiling.
 */
SF_API sf_status sf_gather_rate(int64_t n_rows, int32_t row_bytes, int32_t deg, int32_t reps, int32_t write_rows,
                                void *stream, double *rows_per_s);

#ifdef __cplusplus
}
#endif

#endif /* SPECFILT_H */
