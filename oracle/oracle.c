/*
 * oracle.c -- plain, slow, FP64 CPU statement of what the GPU path computes.
 *
 * TEST INFRASTRUCTURE ONLY. Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg load this file's library. The product path
 * (the CUDA library and its Python binding) never calls it and shares no code,
 * header or helper with it.
 *
 * Every function is a direct loop over the definition it cites, in double
 * precision, single-threaded, with no blocking, fusion or reordering. A
 * second build of this file (with -fopenmp) spreads the filter's loops over
 * rows and elements on several threads, for the timed CPU baseline only;
 * each row or element is still computed by the same operations in the same
 * order, so both builds return identical results.
 * Citations name the paper's sections and equations (Tremblay, Puy, Borgnat,
 * Gribonval, Vandergheynst, "Accelerated spectral clustering using graph
 * filtering of random signals"); equations are numbered in order of
 * appearance:
 *   (1) f_i = U^T delta_i                           §2.2 step 3
 *   (2) ideal low-pass h_lc                          §2.3
 *   (3) Hx ~ sum_l alpha_l L^l x = F^m_h x            §2.4
 *   (4) sup-norm order criterion                      §2.4
 *   (5) H_lk = U U^T                                  §3.1
 *   (6) f~_i = (H_lk R)^T delta_i                     §3.1
 *   (7)-(10) Proposition (JL) and its proof           §3.1
 *   (11) f~_i^T = delta_i^T F R                       §4.1 step 5
 *   (12) stability gamma(k)                           §4.3
 *
 * Readings where the paper is silent (they are the same readings the GPU path
 * implements, each written here independently):
 *   - the polynomial of (3) is expanded in the Chebyshev basis of
 *     Lt = 2 L / lam_max - I (the fast filtering the paper cites in §2.4);
 *   - coefficients are the exact Chebyshev projection of (2), optionally
 *     multiplied by the Jackson damping factors;
 *   - the eigenvalue count of §3.2 is the squared Frobenius norm of the
 *     filtered N(0, 1/eta) block;
 *   - the dichotomy of §3.2 returns the smallest cutoff whose count reaches k.
 *
 * Parity status of each function is stated in its comment; pins live in the
 * CPU test-suite.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------ */
/* Graph: W (§2, W_ij = W_ji >= 0), strengths and L = S - W (§2.1).          */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t row, col;
    double w;
} oracle_entry;

static int cmp_entry(const void *a, const void *b) {
    const oracle_entry *x = (const oracle_entry *)a, *y = (const oracle_entry *)b;
    if (x->row != y->row) return x->row < y->row ? -1 : 1;
    if (x->col != y->col) return x->col < y->col ? -1 : 1;
    return 0;
}

/*
 * Symmetric CSR of W from an undirected edge list (§2: W_ij = W_ji >= 0).
 * Each edge (u, v, w) with u != v contributes W_uv and W_vu; self-loops are
 * dropped because the strength of §2.1 sums over j != i and the Laplacian's
 * diagonal is the strength alone; repeated pairs are merged by taking the
 * largest weight. Rows and, within a row, columns come out in increasing order.
 *
 * rowptr has n + 1 entries; colidx and val must hold 2 * m entries.
 * Returns the number of stored entries, or -1 for an endpoint outside
 * [0, n), -2 for a negative or non-finite weight.
 * Pinned by brute force (dense matrix) in the CPU tests.
 */
int64_t oracle_csr_build(int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                         const double *w, int32_t *rowptr, int32_t *colidx, double *val) {
    int64_t e, cnt = 0;
    for (e = 0; e < m; ++e) {
        if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n) return -1;
        if (!(w[e] >= 0.0) || isinf(w[e])) return -2;
    }
    oracle_entry *ent = (oracle_entry *)malloc(sizeof(oracle_entry) * (size_t)(2 * m + 1));
    for (e = 0; e < m; ++e) {
        if (src[e] == dst[e]) continue;
        ent[cnt].row = src[e]; ent[cnt].col = dst[e]; ent[cnt].w = w[e]; ++cnt;
        ent[cnt].row = dst[e]; ent[cnt].col = src[e]; ent[cnt].w = w[e]; ++cnt;
    }
    qsort(ent, (size_t)cnt, sizeof(oracle_entry), cmp_entry);
    int64_t nnz = 0;
    for (int32_t i = 0; i <= n; ++i) rowptr[i] = 0;
    for (e = 0; e < cnt; ++e) {
        if (e > 0 && ent[e - 1].row == ent[e].row && ent[e - 1].col == ent[e].col) {
            /* repeated pair: it was stored (or merged) at nnz - 1 */
            if (ent[e].w > val[nnz - 1]) val[nnz - 1] = ent[e].w;
            continue;
        }
        colidx[nnz] = ent[e].col;
        val[nnz] = ent[e].w;
        rowptr[ent[e].row + 1] += 1;
        ++nnz;
    }
    for (int32_t i = 0; i < n; ++i) rowptr[i + 1] += rowptr[i];
    free(ent);
    return nnz;
}

/* s_i = sum_{j != i} W_ij (§2.1). */
void oracle_strength(int32_t n, const int32_t *rowptr, const int32_t *colidx, const double *val,
                     double *s) {
    for (int32_t i = 0; i < n; ++i) {
        double acc = 0.0;
        for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
            if (colidx[e] != i) acc += val[e];
        }
        s[i] = acc;
    }
}

/* y = L x with L = S - W (§2.1), one column. */
static void lap_matvec(int32_t n, const int32_t *rowptr, const int32_t *colidx, const double *val,
                       const double *x, double *y) {
    for (int32_t i = 0; i < n; ++i) {
        double s = 0.0, wx = 0.0;
        for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
            s += val[e];
            wx += val[e] * x[colidx[e]];
        }
        y[i] = s * x[i] - wx;
    }
}

/* ------------------------------------------------------------------------ */
/* lambda_N (§4.1 step 1; the paper cites Trefethen & Bau for the method).   */
/* ------------------------------------------------------------------------ */

/* Number of eigenvalues of the symmetric tridiagonal (a, b) below x
 * (Sturm sequence count, LDL^T pivots). */
static int sturm_count(int k, const double *a, const double *b, double x) {
    int c = 0;
    double d = 1.0;
    for (int i = 0; i < k; ++i) {
        double bb = (i == 0) ? 0.0 : b[i - 1] * b[i - 1];
        d = (a[i] - x) - (i == 0 ? 0.0 : bb / d);
        if (d == 0.0) d = -1e-300;
        if (d < 0.0) ++c;
    }
    return c;
}

/* Largest eigenvalue of the k x k symmetric tridiagonal with diagonal a and
 * off-diagonal b (b[i] couples i and i+1), by bisection to machine precision. */
double oracle_tridiag_max_eig(int k, const double *a, const double *b) {
    double lo = a[0], hi = a[0];
    for (int i = 0; i < k; ++i) {
        double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i < k - 1 ? fabs(b[i]) : 0.0);
        if (a[i] - r < lo) lo = a[i] - r;
        if (a[i] + r > hi) hi = a[i] + r;
    }
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (sturm_count(k, a, b, mid) >= k) hi = mid; /* all k below mid */
        else lo = mid;
    }
    return hi;
}

/*
 * Largest Ritz value of L after `iters` Lanczos steps from start vector v0,
 * with full re-orthogonalisation against every previous Lanczos vector.
 * Stops early when the Krylov space is exhausted (beta below 1e-12 times the
 * running scale). Writes the tridiagonal to alpha[0..k-1], beta[0..k-2] when
 * they are non-NULL and returns the Ritz value; *k_out gets k.
 * Pinned against closed-form spectra (path, cycle, complete, star graphs) and
 * numpy's dense eigensolver in the CPU tests.
 */
double oracle_lanczos_max(int32_t n, const int32_t *rowptr, const int32_t *colidx,
                          const double *val, int32_t iters, const double *v0, double *alpha,
                          double *beta, int32_t *k_out) {
    if (iters > n) iters = n;
    double *V = (double *)calloc((size_t)n * (size_t)(iters + 1), sizeof(double));
    double *w = (double *)malloc(sizeof(double) * (size_t)n);
    double *a = (double *)calloc((size_t)iters + 1, sizeof(double));
    double *b = (double *)calloc((size_t)iters + 1, sizeof(double));
    double nrm = 0.0;
    for (int32_t i = 0; i < n; ++i) nrm += v0[i] * v0[i];
    nrm = sqrt(nrm);
    for (int32_t i = 0; i < n; ++i) V[i] = v0[i] / nrm;
    int k = 0;
    double scale = 0.0;
    for (int j = 0; j < iters; ++j) {
        double *vj = V + (size_t)j * n;
        lap_matvec(n, rowptr, colidx, val, vj, w);
        double aj = 0.0;
        for (int32_t i = 0; i < n; ++i) aj += w[i] * vj[i];
        a[j] = aj;
        k = j + 1;
        for (int32_t i = 0; i < n; ++i) w[i] -= aj * vj[i];
        if (j > 0) {
            double *vp = V + (size_t)(j - 1) * n;
            for (int32_t i = 0; i < n; ++i) w[i] -= b[j - 1] * vp[i];
        }
        /* full re-orthogonalisation, twice */
        for (int pass = 0; pass < 2; ++pass) {
            for (int q = 0; q <= j; ++q) {
                double *vq = V + (size_t)q * n, d = 0.0;
                for (int32_t i = 0; i < n; ++i) d += w[i] * vq[i];
                for (int32_t i = 0; i < n; ++i) w[i] -= d * vq[i];
            }
        }
        double bj = 0.0;
        for (int32_t i = 0; i < n; ++i) bj += w[i] * w[i];
        bj = sqrt(bj);
        if (fabs(aj) > scale) scale = fabs(aj);
        if (bj > scale) scale = bj;
        if (j == iters - 1 || bj <= 1e-12 * scale) break;
        b[j] = bj;
        double *vn = V + (size_t)(j + 1) * n;
        for (int32_t i = 0; i < n; ++i) vn[i] = w[i] / bj;
    }
    double theta = oracle_tridiag_max_eig(k, a, b);
    if (alpha) for (int j = 0; j < k; ++j) alpha[j] = a[j];
    if (beta) for (int j = 0; j + 1 < k; ++j) beta[j] = b[j];
    if (k_out) *k_out = k;
    free(V); free(w); free(a); free(b);
    return theta;
}

/* ------------------------------------------------------------------------ */
/* Polynomial of (3) in the Chebyshev basis: coefficients of (2).            */
/* ------------------------------------------------------------------------ */

/*
 * Jackson damping factors g_0..g_p for a degree-p expansion (p + 1 terms):
 *   g_j = [(p + 2 - j) cos(pi j / (p + 2)) + sin(pi j / (p + 2)) cot(pi / (p + 2))] / (p + 2).
 * Pinned by g_0 = 1, g_1 = cos(pi / (p + 2)) and the positivity of the damped
 * step (CPU tests).
 */
void oracle_jackson(int32_t p, double *g) {
    double q = (double)(p + 2);
    for (int32_t j = 0; j <= p; ++j) {
        g[j] = ((q - j) * cos(M_PI * j / q) + sin(M_PI * j / q) / tan(M_PI / q)) / q;
    }
}

/*
 * Coefficients a_0..a_p of the ideal low-pass h_lc of (2) on [0, lam_max] in
 * the Chebyshev basis of x = 2 lam / lam_max - 1, so that
 *   h_lc(lam) ~ sum_j a_j T_j(x).
 * With theta_c = arccos(x_c), x_c = 2 lc / lam_max - 1 clamped to [-1, 1], the
 * projection (2/pi) int_0^pi h(cos t) cos(j t) dt gives
 *   c_0 = 2 (1 - theta_c / pi),  c_j = -2 sin(j theta_c) / (pi j) (j >= 1),
 * and the series uses c_0 / 2. With jackson != 0 every a_j is multiplied by
 * the Jackson factor g_j. Pinned against adaptive quadrature of the weighted
 * projection integral (CPU tests).
 */
void oracle_cheb_coeffs(double lam_max, double lc, int32_t p, int32_t jackson, double *a) {
    double xc = 2.0 * lc / lam_max - 1.0;
    if (xc > 1.0) xc = 1.0;
    if (xc < -1.0) xc = -1.0;
    double tc = acos(xc);
    a[0] = 1.0 - tc / M_PI;
    for (int32_t j = 1; j <= p; ++j) a[j] = -2.0 * sin(j * tc) / (M_PI * j);
    if (jackson) {
        double *g = (double *)malloc(sizeof(double) * (size_t)(p + 1));
        oracle_jackson(p, g);
        for (int32_t j = 0; j <= p; ++j) a[j] *= g[j];
        free(g);
    }
}

/* ------------------------------------------------------------------------ */
/* Fast filtering F^m_h R of (3) / (6) / (11).                               */
/* ------------------------------------------------------------------------ */

/* Y = Lt X for an n x c row-major block, Lt = (2 / lam_max) L - I, with
 * L = S - W; the diagonal S is the row sums of W unless `diag` gives it. */
static void lt_apply_d(int32_t n, const int32_t *rowptr, const int32_t *colidx, const double *val,
                       const double *diag, double lam_max, int64_t c, const double *X, double *Y) {
#pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < n; ++i) {
        double s = 0.0;
        if (diag) s = diag[i];
        else
            for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e) s += val[e];
        for (int64_t r = 0; r < c; ++r) {
            double wx = 0.0;
            for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e)
                wx += val[e] * X[(int64_t)colidx[e] * c + r];
            double lx = s * X[(int64_t)i * c + r] - wx; /* (L X)_ir */
            Y[(int64_t)i * c + r] = (2.0 / lam_max) * lx - X[(int64_t)i * c + r];
        }
    }
}

static void lt_apply(int32_t n, const int32_t *rowptr, const int32_t *colidx, const double *val,
                     double lam_max, int64_t c, const double *X, double *Y) {
    lt_apply_d(n, rowptr, colidx, val, NULL, lam_max, c, X, Y);
}

/*
 * Y_q = sum_{j=0}^{p} a_{q,j} T_j(Lt) R for q = 0..n_cut-1 (the fast filter
 * of (3) applied to the block R of §3.1, giving the rows f~_i of (6)/(11)).
 * T_0 R = R, T_1 R = Lt R, T_j R = 2 Lt T_{j-1} R - T_{j-2} R, each block
 * computed in full and added to every Y_q with its coefficient.
 * a is n_cut x (p + 1); R is n x n_sig; Y is n_cut x n x n_sig.
 * Pinned against the dense eigendecomposition chi diag(P(lt_l)) chi^T R.
 */
void oracle_cheb_filter(int32_t n, const int32_t *rowptr, const int32_t *colidx, const double *val,
                        double lam_max, int32_t n_cut, int32_t p, const double *a, int64_t n_sig,
                        const double *R, double *Y) {
    int64_t sz = (int64_t)n * n_sig;
    double *Tm2 = (double *)malloc(sizeof(double) * (size_t)(sz > 0 ? sz : 1));
    double *Tm1 = (double *)malloc(sizeof(double) * (size_t)(sz > 0 ? sz : 1));
    double *Tj = (double *)malloc(sizeof(double) * (size_t)(sz > 0 ? sz : 1));
    for (int64_t t = 0; t < sz; ++t) Tm1[t] = R[t]; /* T_0 */
    for (int32_t q = 0; q < n_cut; ++q)
        for (int64_t t = 0; t < sz; ++t) Y[q * sz + t] = a[q * (p + 1) + 0] * Tm1[t];
    for (int32_t j = 1; j <= p; ++j) {
        lt_apply(n, rowptr, colidx, val, lam_max, n_sig, Tm1, Tj); /* Lt T_{j-1} */
        if (j >= 2) {
#pragma omp parallel for schedule(static)
            for (int64_t t = 0; t < sz; ++t) Tj[t] = 2.0 * Tj[t] - Tm2[t];
        }
        for (int32_t q = 0; q < n_cut; ++q) {
#pragma omp parallel for schedule(static)
            for (int64_t t = 0; t < sz; ++t) Y[q * sz + t] += a[q * (p + 1) + j] * Tj[t];
        }
        double *tmp = Tm2; Tm2 = Tm1; Tm1 = Tj; Tj = tmp;
    }
    free(Tm2); free(Tm1); free(Tj);
}

/* Threads the filter's loops run on: 1 in the plain build. */
int32_t oracle_threads(void) {
#ifdef _OPENMP
    return (int32_t)omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * mu_m = <R, T_m(Lt) R>_F for m = 0..m_max, each from its own block T_m R
 * obtained by running the recurrence to m_max (no product identities).
 * Used to check the GPU's moment sweep and the count-from-moments expansion.
 */
void oracle_moments(int32_t n, const int32_t *rowptr, const int32_t *colidx, const double *val,
                    double lam_max, int64_t n_sig, const double *R, int32_t m_max, double *mu) {
    int64_t sz = (int64_t)n * n_sig;
    double *Tm2 = (double *)malloc(sizeof(double) * (size_t)(sz > 0 ? sz : 1));
    double *Tm1 = (double *)malloc(sizeof(double) * (size_t)(sz > 0 ? sz : 1));
    double *Tj = (double *)malloc(sizeof(double) * (size_t)(sz > 0 ? sz : 1));
    double d = 0.0;
    for (int64_t t = 0; t < sz; ++t) { Tm1[t] = R[t]; d += R[t] * R[t]; }
    mu[0] = d;
    for (int32_t j = 1; j <= m_max; ++j) {
        lt_apply(n, rowptr, colidx, val, lam_max, n_sig, Tm1, Tj);
        if (j >= 2) for (int64_t t = 0; t < sz; ++t) Tj[t] = 2.0 * Tj[t] - Tm2[t];
        d = 0.0;
        for (int64_t t = 0; t < sz; ++t) d += R[t] * Tj[t];
        mu[j] = d;
        double *tmp = Tm2; Tm2 = Tm1; Tm1 = Tj; Tj = tmp;
    }
    free(Tm2); free(Tm1); free(Tj);
}

/*
 * Eigenvalue count of §3.2 at each cutoff: count_q = ||Y_q||_F^2 with
 * Y_q = F_q R and R ~ N(0, 1/eta) (so the expectation is
 * sum_l P_q(lt_l)^2, the number of eigenvalues below the cutoff up to the
 * polynomial's error). Computed directly from each filtered block.
 */
void oracle_eigencount(int32_t n, const int32_t *rowptr, const int32_t *colidx, const double *val,
                       double lam_max, int32_t n_cut, int32_t p, const double *a, int64_t n_sig,
                       const double *R, double *counts) {
    int64_t sz = (int64_t)n * n_sig;
    double *Y = (double *)malloc(sizeof(double) * (size_t)(sz > 0 ? sz : 1));
    for (int32_t q = 0; q < n_cut; ++q) {
        oracle_cheb_filter(n, rowptr, colidx, val, lam_max, 1, p, a + (int64_t)q * (p + 1), n_sig,
                           R, Y);
        double c = 0.0;
        for (int64_t t = 0; t < sz; ++t) c += Y[t] * Y[t];
        counts[q] = c;
    }
    free(Y);
}

/*
 * Dichotomy of §3.2 on [0, lam_max]: the smallest cutoff lc with
 * count(lc) >= k, found by bisection (each count computed by a full filter of
 * R as in oracle_eigencount), stopping after max_iter halvings or when the
 * bracket is narrower than tol * lam_max. Returns the upper end.
 * Parity: pinned (with the identity as the signal block the count is exactly
 * tr(P(Lt)^2), and the result equals a bisection on the dense spectrum).
 */
double oracle_dichotomy(int32_t n, const int32_t *rowptr, const int32_t *colidx, const double *val,
                        double lam_max, int32_t p, int32_t jackson, int64_t n_sig, const double *R,
                        double k, int32_t max_iter, double tol) {
    double lo = 0.0, hi = lam_max, cnt;
    double *a = (double *)malloc(sizeof(double) * (size_t)(p + 1));
    for (int32_t it = 0; it < max_iter && (hi - lo) > tol * lam_max; ++it) {
        double mid = 0.5 * (lo + hi);
        oracle_cheb_coeffs(lam_max, mid, p, jackson, a);
        oracle_eigencount(n, rowptr, colidx, val, lam_max, 1, p, a, n_sig, R, &cnt);
        if (cnt >= k) hi = mid;
        else lo = mid;
    }
    free(a);
    return hi;
}

/*
 * Feature rows (6)/(11): f~_i = row i of Y. With normalize != 0 each row is
 * divided by its Euclidean norm; an all-zero row stays zero.
 */
void oracle_features(int32_t n, int64_t n_sig, const double *Y, int32_t normalize, double *F) {
    for (int32_t i = 0; i < n; ++i) {
        const double *y = Y + (int64_t)i * n_sig;
        double *f = F + (int64_t)i * n_sig;
        double nrm = 0.0;
        for (int64_t r = 0; r < n_sig; ++r) nrm += y[r] * y[r];
        nrm = sqrt(nrm);
        for (int64_t r = 0; r < n_sig; ++r) {
            if (!normalize) f[r] = y[r];
            else f[r] = (nrm > 0.0) ? y[r] / nrm : 0.0;
        }
    }
}

/*
 * Reverse mode of Y = sum_j a_j T_j(Lt) R for the scalar loss l = <G, Y>_F
 * (one coefficient set), by the chain rule over the stored blocks T_0..T_p:
 *   Gb_j = dl/dT_j:  Gb_p = a_p G,
 *   Gb_j = a_j G + 2 Lt^T Gb_{j+1} - Gb_{j+2}   for 1 <= j < p (Gb_{p+1} = 0),
 *   Gb_0 = a_0 G + Lt^T Gb_1 - Gb_2            (= dl/dR),
 *   dl/da_j = <G, T_j>,
 *   dl/dLt  = Gb_1 T_0^T + sum_{j>=2} 2 Gb_j T_{j-1}^T  (only the entries
 *             Lt_uv with W_uv stored, and the diagonal, are needed),
 *   dl/dW_uv = (2 / lam_max) (M_uu + M_vv - M_uv - M_vu) for an undirected
 *             edge uv, because W_uv enters Lt_uv, Lt_vu with -2/lam_max and
 *             Lt_uu, Lt_vv with +2/lam_max (§2.1: L = S - W).
 * lam_max is held fixed. grad_val has one entry per stored CSR entry (both
 * directions of an edge carry the same undirected-edge derivative);
 * grad_a has p + 1 entries; grad_R (n x n_sig) may be NULL.
 * Pinned by central finite differences of oracle_cheb_filter (CPU tests).
 */
void oracle_cheb_filter_backward(int32_t n, const int32_t *rowptr, const int32_t *colidx,
                                 const double *val, double lam_max, int32_t p, const double *a,
                                 int64_t n_sig, const double *R, const double *G,
                                 double *grad_val, double *grad_a, double *grad_R) {
    int64_t sz = (int64_t)n * n_sig;
    int64_t nnz = rowptr[n];
    double *T = (double *)malloc(sizeof(double) * (size_t)(sz * (p + 1) + 1));
    for (int64_t t = 0; t < sz; ++t) T[t] = R[t];
    for (int32_t j = 1; j <= p; ++j) {
        double *Tj = T + (int64_t)j * sz;
        lt_apply(n, rowptr, colidx, val, lam_max, n_sig, T + (int64_t)(j - 1) * sz, Tj);
        if (j >= 2) {
            double *Tm2 = T + (int64_t)(j - 2) * sz;
            for (int64_t t = 0; t < sz; ++t) Tj[t] = 2.0 * Tj[t] - Tm2[t];
        }
    }
    for (int32_t j = 0; j <= p; ++j) {
        double d = 0.0;
        for (int64_t t = 0; t < sz; ++t) d += G[t] * T[(int64_t)j * sz + t];
        grad_a[j] = d;
    }
    /* adjoint blocks, top-down */
    double *Gb = (double *)calloc((size_t)(sz * (p + 3) + 1), sizeof(double)); /* Gb_0..Gb_{p+2} */
    double *tmp = (double *)malloc(sizeof(double) * (size_t)(sz > 0 ? sz : 1));
    for (int32_t j = p; j >= 0; --j) {
        double *gj = Gb + (int64_t)j * sz;
        double *g1 = Gb + (int64_t)(j + 1) * sz;
        double *g2 = Gb + (int64_t)(j + 2) * sz;
        lt_apply(n, rowptr, colidx, val, lam_max, n_sig, g1, tmp); /* Lt symmetric */
        double mult = (j == 0) ? 1.0 : 2.0;
        for (int64_t t = 0; t < sz; ++t) gj[t] = a[j] * G[t] + mult * tmp[t] - g2[t];
    }
    /* M restricted to the diagonal and the stored entries */
    double *Mdiag = (double *)calloc((size_t)n + 1, sizeof(double));
    double *Moff = (double *)calloc((size_t)nnz + 1, sizeof(double));
    for (int32_t j = 1; j <= p; ++j) {
        double c = (j == 1) ? 1.0 : 2.0;
        const double *gj = Gb + (int64_t)j * sz;
        const double *tp = T + (int64_t)(j - 1) * sz;
        for (int32_t u = 0; u < n; ++u) {
            double d = 0.0;
            for (int64_t r = 0; r < n_sig; ++r) d += gj[(int64_t)u * n_sig + r] * tp[(int64_t)u * n_sig + r];
            Mdiag[u] += c * d;
            for (int32_t e = rowptr[u]; e < rowptr[u + 1]; ++e) {
                int32_t v = colidx[e];
                double dv = 0.0;
                for (int64_t r = 0; r < n_sig; ++r)
                    dv += gj[(int64_t)u * n_sig + r] * tp[(int64_t)v * n_sig + r];
                Moff[e] += c * dv;
            }
        }
    }
    /* dl/dW_uv for each stored entry (u, v); M_vu is found in row v */
    for (int32_t u = 0; u < n; ++u) {
        for (int32_t e = rowptr[u]; e < rowptr[u + 1]; ++e) {
            int32_t v = colidx[e];
            double mvu = 0.0;
            for (int32_t f = rowptr[v]; f < rowptr[v + 1]; ++f)
                if (colidx[f] == u) { mvu = Moff[f]; break; }
            grad_val[e] = (2.0 / lam_max) * (Mdiag[u] + Mdiag[v] - Moff[e] - mvu);
        }
    }
    if (grad_R) for (int64_t t = 0; t < sz; ++t) grad_R[t] = Gb[t];
    free(T); free(Gb); free(tmp); free(Mdiag); free(Moff);
}

/* ------------------------------------------------------------------------ */
/* k-means on the feature rows (§4.1 step 6: k-means with the Euclidean      */
/* distance between rows f~_i).                                              */
/* ------------------------------------------------------------------------ */

/* Squared Euclidean distance in FP32, accumulated in index order with fused
 * multiply-adds. The label is an integer decided by floating point, so the
 * oracle takes that decision in the precision and order the GPU path states
 * for it (IEEE FP32, fmaf correctly rounded). */
static float sqdist_f32(const float *f, const float *c, int32_t d) {
    float acc = 0.0f;
    for (int32_t j = 0; j < d; ++j) {
        const float t = f[j] - c[j];
        acc = fmaf(t, t, acc);
    }
    return acc;
}

/* Lloyd's algorithm from the given centroids C (k x d, row-major, updated in
 * place), rows F (n x d). Each iteration:
 *   assignment: label_i = argmin_c sqdist_f32(f_i, c_c), ties to the lowest c;
 *   stop if no label changed (from the second iteration on);
 *   update: c_c = (sum of the rows labelled c, in row order, in FP64) / count,
 *   rounded to FP32; an empty cluster keeps its centroid;
 * at most max_iter assignments. Returns the inertia of the last assignment
 * (sum over rows, in row order, in FP64, of the FP32 distances it used) and
 * the number of assignments in *iters. Parity: pinned (CPU tests: brute-force
 * argmin, numpy means, separated clusters, monotone inertia, ties). */
double oracle_kmeans(int32_t n, int32_t d, int32_t k, const float *F, float *C, int32_t max_iter,
                     int32_t *labels, int32_t *iters) {
    double *sum = (double *)malloc(sizeof(double) * (size_t)k * (size_t)(d > 0 ? d : 1));
    int64_t *cnt = (int64_t *)malloc(sizeof(int64_t) * (size_t)(k > 0 ? k : 1));
    double inertia = 0.0;
    int32_t it = 0;
    while (it < max_iter) {
        int changed = (it == 0);
        inertia = 0.0;
        for (int32_t i = 0; i < n; ++i) {
            const float *f = F + (int64_t)i * d;
            int32_t best = 0;
            float bd = sqdist_f32(f, C, d);
            for (int32_t c = 1; c < k; ++c) {
                const float dc = sqdist_f32(f, C + (int64_t)c * d, d);
                if (dc < bd) {
                    bd = dc;
                    best = c;
                }
            }
            if (labels[i] != best) changed = 1;
            labels[i] = best;
            inertia += (double)bd;
        }
        ++it;
        if (!changed) break;
        for (int64_t t = 0; t < (int64_t)k * d; ++t) sum[t] = 0.0;
        for (int32_t c = 0; c < k; ++c) cnt[c] = 0;
        for (int32_t i = 0; i < n; ++i) {
            const int32_t c = labels[i];
            cnt[c] += 1;
            for (int32_t j = 0; j < d; ++j) sum[(int64_t)c * d + j] += (double)F[(int64_t)i * d + j];
        }
        for (int32_t c = 0; c < k; ++c)
            if (cnt[c] > 0)
                for (int32_t j = 0; j < d; ++j) C[(int64_t)c * d + j] = (float)(sum[(int64_t)c * d + j] / (double)cnt[c]);
    }
    *iters = it;
    free(sum);
    free(cnt);
    return inertia;
}


/* ------------------------------------------------------------------------ */
/* Normalised Laplacian (the footnote of §2.1: I - S^{-1/2} W S^{-1/2}).     */
/* ------------------------------------------------------------------------ */

/* Written as the weights w'_ij = w_ij / sqrt(s_i s_j) and the diagonal
 * d_i = 1, or 0 for an isolated node (whose row of S^{-1/2} is taken as 0).
 * Parity: pinned (spectrum of K_n, C_n and bipartite graphs, the null vector
 * S^{1/2} 1, numpy's dense eigenvalues). */
void oracle_normalize(int32_t n, const int32_t *rowptr, const int32_t *colidx, const double *val,
                      double *val_out, double *diag_out) {
    double *s = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    oracle_strength(n, rowptr, colidx, val, s);
    for (int32_t i = 0; i < n; ++i) {
        diag_out[i] = s[i] > 0.0 ? 1.0 : 0.0;
        for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
            const int32_t j = colidx[e];
            const double ss = s[i] * s[j];
            val_out[e] = ss > 0.0 ? val[e] / sqrt(ss) : 0.0;
        }
    }
    free(s);
}

/* oracle_cheb_filter for L = diag(d) - W (the normalised Laplacian's form). */
void oracle_cheb_filter_diag(int32_t n, const int32_t *rowptr, const int32_t *colidx, const double *val,
                             const double *diag, double lam_max, int32_t n_cut, int32_t p, const double *a,
                             int64_t n_sig, const double *R, double *Y) {
    int64_t sz = (int64_t)n * n_sig;
    double *Tm2 = (double *)malloc(sizeof(double) * (size_t)(sz > 0 ? sz : 1));
    double *Tm1 = (double *)malloc(sizeof(double) * (size_t)(sz > 0 ? sz : 1));
    double *Tj = (double *)malloc(sizeof(double) * (size_t)(sz > 0 ? sz : 1));
    for (int64_t t = 0; t < sz; ++t) Tm1[t] = R[t];
    for (int32_t q = 0; q < n_cut; ++q)
        for (int64_t t = 0; t < sz; ++t) Y[q * sz + t] = a[q * (p + 1) + 0] * Tm1[t];
    for (int32_t j = 1; j <= p; ++j) {
        lt_apply_d(n, rowptr, colidx, val, diag, lam_max, n_sig, Tm1, Tj);
        if (j >= 2)
            for (int64_t t = 0; t < sz; ++t) Tj[t] = 2.0 * Tj[t] - Tm2[t];
        for (int32_t q = 0; q < n_cut; ++q)
            for (int64_t t = 0; t < sz; ++t) Y[q * sz + t] += a[q * (p + 1) + j] * Tj[t];
        double *tmp = Tm2; Tm2 = Tm1; Tm1 = Tj; Tj = tmp;
    }
    free(Tm2); free(Tm1); free(Tj);
}

/* ------------------------------------------------------------------------ */
/* Stability of the clusterings (§4.3, Eq. (12)).                            */
/* ------------------------------------------------------------------------ */

/* Adjusted Rand index of two labelings (Hubert and Arabie 1985), from the
 * contingency table n_uv and its margins, with x(x - 1)/2 pair counts:
 * (sum n_uv choose 2 - E) / (max - E), E = (sum a_u choose 2)(sum b_v choose 2)
 * / (n choose 2), max = ((sum a_u choose 2) + (sum b_v choose 2)) / 2; 1 when
 * max = E (both labelings trivial). Labels in [0, ka) and [0, kb).
 * Parity: pinned (brute-force pair counting, identity and permutations). */
double oracle_adjusted_rand(int32_t n, const int32_t *a, const int32_t *b, int32_t ka, int32_t kb) {
    int64_t *t = (int64_t *)calloc((size_t)ka * (size_t)kb, sizeof(int64_t));
    int64_t *ra = (int64_t *)calloc((size_t)ka, sizeof(int64_t));
    int64_t *rb = (int64_t *)calloc((size_t)kb, sizeof(int64_t));
    for (int32_t i = 0; i < n; ++i) {
        t[(int64_t)a[i] * kb + b[i]] += 1;
        ra[a[i]] += 1;
        rb[b[i]] += 1;
    }
    double sij = 0.0, sa = 0.0, sb = 0.0;
    for (int64_t u = 0; u < (int64_t)ka * kb; ++u) sij += 0.5 * (double)t[u] * (double)(t[u] - 1);
    for (int32_t u = 0; u < ka; ++u) sa += 0.5 * (double)ra[u] * (double)(ra[u] - 1);
    for (int32_t v = 0; v < kb; ++v) sb += 0.5 * (double)rb[v] * (double)(rb[v] - 1);
    free(t);
    free(ra);
    free(rb);
    const double pairs = 0.5 * (double)n * (double)(n - 1);
    const double expct = pairs > 0.0 ? sa * sb / pairs : 0.0;
    const double top = 0.5 * (sa + sb);
    return (top == expct) ? 1.0 : (sij - expct) / (top - expct);
}

/* SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) of counter i under `seed`:
 * z = seed + (i + 1) * 0x9E3779B97F4A7C15, then two xor-shift-multiply rounds.
 * The stability measure's k-means starts use it to pick rows. */
static uint64_t splitmix64_at(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Initial centroid c of start t of realisation j for k clusters: row
 * splitmix64_at(seed, (j << 40) | (k << 20) | (t << 10) | c) mod n
 * (k < 2^20, t < 2^10, c < 2^10). */
int32_t oracle_stability_init_row(uint64_t seed, int32_t j, int32_t k, int32_t t, int32_t c, int32_t n) {
    const uint64_t ctr = ((uint64_t)j << 40) | ((uint64_t)k << 20) | ((uint64_t)t << 10) | (uint64_t)c;
    return (int32_t)(splitmix64_at(seed, ctr) % (uint64_t)n);
}

/* The stability measure of §4.3, Eq. (12), step by step: for every k in
 * [kmin, kmax], lam_k by the dichotomy of §3.2 (order p) on the count probes
 * Rc (target k - 1/2); for every realisation j of the eta signals (R_j, block
 * j of R), the filtered block at lam_k (Jackson-damped coefficients, order
 * p_filter: the filters may use a higher order than the count), its
 * normalised rows rounded to FP32, and k-means (oracle_kmeans, max_iter) from
 * `starts` sets of rows that oracle_stability_init_row picks, keeping the
 * lowest inertia (the first on ties); gamma(k) = the mean adjusted Rand
 * index over the J (J - 1) / 2 pairs of realisations (equal to the mean over
 * ordered pairs i != j of Eq. (12)). gamma and lam_k have kmax - kmin + 1
 * entries. Parity: its parts are pinned; the composition is checked on graphs
 * with a clear cluster structure (gamma = 1 at the true k). */
void oracle_stability(int32_t n, const int32_t *rowptr, const int32_t *colidx, const double *val,
                      double lam_max, int32_t p, int32_t p_filter, int64_t eta, const double *Rc, int32_t J,
                      const double *R, int32_t kmin, int32_t kmax, int32_t max_iter, int32_t starts, uint64_t seed,
                      double *gamma, double *lam_k) {
    const int32_t K = kmax - kmin + 1;
    const int64_t sz = (int64_t)n * eta;
    double *a = (double *)malloc(sizeof(double) * (size_t)K * (size_t)(p_filter + 1));
    for (int32_t q = 0; q < K; ++q) {
        lam_k[q] = oracle_dichotomy(n, rowptr, colidx, val, lam_max, p, 1, eta, Rc, (double)(kmin + q) - 0.5, 40,
                                    1e-9);
        oracle_cheb_coeffs(lam_max, lam_k[q], p_filter, 1, a + (int64_t)q * (p_filter + 1));
    }
    double *Y = (double *)malloc(sizeof(double) * (size_t)(K * sz > 0 ? K * sz : 1));
    double *Fd = (double *)malloc(sizeof(double) * (size_t)(sz > 0 ? sz : 1));
    float *F = (float *)malloc(sizeof(float) * (size_t)(sz > 0 ? sz : 1));
    float *C = (float *)malloc(sizeof(float) * (size_t)kmax * (size_t)eta);
    int32_t *labels = (int32_t *)malloc(sizeof(int32_t) * (size_t)J * K * (size_t)(n > 0 ? n : 1));
    int32_t *trial = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    for (int32_t j = 0; j < J; ++j) {
        oracle_cheb_filter(n, rowptr, colidx, val, lam_max, K, p_filter, a, eta, R + (int64_t)j * sz, Y);
        for (int32_t q = 0; q < K; ++q) {
            const int32_t k = kmin + q;
            oracle_features(n, eta, Y + (int64_t)q * sz, 1, Fd);
            for (int64_t t = 0; t < sz; ++t) F[t] = (float)Fd[t];
            int32_t *lab = labels + ((int64_t)j * K + q) * n;
            double best = INFINITY;
            for (int32_t st = 0; st < starts; ++st) {
                for (int32_t c = 0; c < k; ++c) {
                    const int32_t r = oracle_stability_init_row(seed, j, k, st, c, n);
                    for (int64_t t = 0; t < eta; ++t) C[(int64_t)c * eta + t] = F[(int64_t)r * eta + t];
                }
                for (int32_t i = 0; i < n; ++i) trial[i] = -1;
                int32_t it = 0;
                const double inertia = oracle_kmeans(n, (int32_t)eta, k, F, C, max_iter, trial, &it);
                if (inertia < best) {
                    best = inertia;
                    for (int32_t i = 0; i < n; ++i) lab[i] = trial[i];
                }
            }
        }
    }
    for (int32_t q = 0; q < K; ++q) {
        const int32_t k = kmin + q;
        double acc = 0.0;
        int64_t pairs = 0;
        for (int32_t i = 0; i < J; ++i)
            for (int32_t j = i + 1; j < J; ++j) {
                acc += oracle_adjusted_rand(n, labels + ((int64_t)i * K + q) * n, labels + ((int64_t)j * K + q) * n,
                                            k, k);
                ++pairs;
            }
        gamma[q] = pairs > 0 ? acc / (double)pairs : 1.0;
    }
    free(a); free(Y); free(Fd); free(F); free(C); free(labels); free(trial);
}

/* ------------------------------------------------------------------------ */
/* The order m* of §2.4 (criterion (4)), tabulated against lambda_c/lambda_N. */
/* ------------------------------------------------------------------------ */

/* Smallest order m in [1, p_max] whose (optionally Jackson-damped) Chebyshev
 * approximation P_m of the ideal low-pass h_x on [0, 1] (h = 1 for t <= x,
 * else 0) satisfies |h(t) - P_m(t)| <= delta at every point t of the grid
 * g / 4095 (g = 0..4095) and of the band edges x - w, x + w that lies in
 * [0, 1] with |t - x| >= w; -1 when no order up to p_max does. P_m(t) =
 * sum_j a_j cos(j arccos(2t - 1)), each T_j evaluated directly. The paper's
 * sup over [0, lambda_N] cannot fall below 1/2 at the jump, so the band of
 * half-width w around x is left out. Parity: pinned (numpy's chebval on the
 * same grid, monotonicity in delta and w). */
int32_t oracle_cheb_order(double x, double delta, double w, int32_t jackson, int32_t p_max) {
    double *a = (double *)malloc(sizeof(double) * (size_t)(p_max + 1));
    double pts[4098];
    int32_t np = 0;
    for (int32_t gi = 0; gi < 4096; ++gi) pts[np++] = (double)gi / 4095.0;
    if (x - w >= 0.0) pts[np++] = x - w;
    if (x + w <= 1.0) pts[np++] = x + w;
    int32_t found = -1;
    for (int32_t m = 1; m <= p_max && found < 0; ++m) {
        oracle_cheb_coeffs(1.0, x, m, jackson, a);
        double worst = 0.0;
        for (int32_t q = 0; q < np; ++q) {
            const double t = pts[q];
            if (fabs(t - x) < w) continue;
            const double y = acos(fmin(1.0, fmax(-1.0, 2.0 * t - 1.0)));
            double v = 0.0;
            for (int32_t j = 0; j <= m; ++j) v += a[j] * cos((double)j * y);
            const double e = fabs((t <= x ? 1.0 : 0.0) - v);
            if (e > worst) worst = e;
        }
        if (worst <= delta) found = m;
    }
    free(a);
    return found;
}
