/*
 * CPU oracle for the stochastic Chebyshev log-determinant estimator
 * (Han, Malioutov, Shin, "Large-scale Log-determinant Computation through
 * Stochastic Chebyshev Expansions", arXiv 1503.06394).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct
 * FP64 reference that the GPU library is checked against.  Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg may load it.  It shares
 * no code, header, table or constant generator with the CUDA library, and the
 * library never calls it.
 *
 * Everything here is FP64 and follows the paper's definitions in the paper's
 * order, with no blocking, fusion or reordering:
 *   - Philox4x32-10 counter-based generator (Salmon et al., SC'11), used to
 *     draw the Rademacher probes of Sec. 2.2;
 *   - Chebyshev interpolation coefficients at first-kind nodes (Sec. 2.1);
 *   - the Chebyshev-Hutchinson estimator of Algorithm 1, in the general
 *     spectral-interval form (Sec. 4.1, map g) and in the literal form;
 *   - Algorithm 2 for general non-singular C (log|det C| = 1/2 logdet C^T C);
 *   - Gershgorin bounds and the norm bound sigma_max <= sqrt(||C||_1 ||C||_inf)
 *     (Sec. 3.2);
 *   - dense Cholesky log-determinant 2 sum log L_ii (Sec. 1);
 *   - the exact gradient of the estimator with respect to the stored values
 *     (an extension: reverse-mode differentiation of the recurrence of
 *     Sec. 2.2, written as the plain sum over degrees of the chain rule).
 *
 * Pins (what checks this file against something other than itself) live in
 * tests/test_oracle_*.py; the Philox stream is pinned against cuRAND's host
 * Philox4_32_10 generator and by statistics.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define EXPORT __attribute__((visibility("default")))

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as    */
/* easy as 1, 2, 3", SC'11).  One round maps the counter (c0,c1,c2,c3) with    */
/* key (k0,k1) to (hi(M1*c2)^c1^k0, lo(M1*c2), hi(M0*c0)^c3^k1, lo(M0*c0));    */
/* the key is bumped by the Weyl constants between rounds; ten rounds.         */
/* ------------------------------------------------------------------------- */
EXPORT void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                                 uint32_t out[4]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0; k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Rademacher entry v[i,p] in {+1,-1} (Sec. 2.2, Pr(+1)=Pr(-1)=1/2).  The paper
 * does not say how the signs are drawn; the stream is fixed as: key = seed
 * (low word, high word); counter = (i low word, i high word, p / 128, 0);
 * sign bit = bit (p mod 32) of output word ((p / 32) mod 4); v = 1 - 2*bit. */
EXPORT double oracle_rademacher(uint64_t seed, int64_t i, int64_t p) {
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint64_t ui = (uint64_t)i;
    uint32_t ctr[4] = {(uint32_t)ui, (uint32_t)(ui >> 32), (uint32_t)(p / 128), 0u};
    uint32_t out[4];
    oracle_philox4x32_10(ctr, key, out);
    uint32_t word = out[(p / 32) % 4];
    uint32_t bit = (word >> (p % 32)) & 1u;
    return bit ? -1.0 : 1.0;
}

/* Fills V (d x nprobe, row-major, probe index fastest) with v[i, probes[q]]. */
EXPORT void oracle_rademacher_fill(uint64_t seed, int64_t d, const int64_t* probes,
                                   int64_t nprobe, double* V) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < d; ++i)
        for (int64_t q = 0; q < nprobe; ++q)
            V[i * nprobe + q] = oracle_rademacher(seed, i, probes[q]);
}

/* ------------------------------------------------------------------------- */
/* Chebyshev interpolation (Sec. 2.1).  For f on [-1,1] the degree-n           */
/* interpolant is p_n = sum_j c_j T_j with                                     */
/*   c_0 = 1/(n+1) sum_k f(x_k) T_0(x_k),  c_j = 2/(n+1) sum_k f(x_k) T_j(x_k), */
/*   x_k = cos(pi (k + 1/2) / (n+1)),  k = 0..n.                              */
/* Here f(x) = log( ((b-a) x + a + b) / 2 ): the logarithm on [a,b] pulled     */
/* back to [-1,1] by the affine map of Sec. 4.1.                               */
/* ------------------------------------------------------------------------- */
static double log_on_interval(double x, double a, double b) {
    return log(((b - a) * x + a + b) / 2.0);
}

/* T_j(x) by the three-term recurrence of Eq. (chebreq). */
static double cheb_T(int j, double x) {
    if (j == 0) return 1.0;
    double tm1 = 1.0, t = x;
    for (int i = 1; i < j; ++i) {
        double tp1 = 2.0 * x * t - tm1;
        tm1 = t;
        t = tp1;
    }
    return t;
}

EXPORT void oracle_cheb_coeffs(int n, double a, double b, double* c) {
    for (int j = 0; j <= n; ++j) {
        double s = 0.0;
        for (int k = 0; k <= n; ++k) {
            double xk = cos(M_PI * (k + 0.5) / (n + 1));
            s += log_on_interval(xk, a, b) * cheb_T(j, xk);
        }
        c[j] = (j == 0 ? 1.0 : 2.0) / (n + 1) * s;
    }
}

/* Same nodes formula for the literal Algorithm 1 function
 * f(x) = log(1 - ((1 - 2 delta) x + 1) / 2). */
EXPORT void oracle_cheb_coeffs_alg1(int n, double delta, double* c) {
    for (int j = 0; j <= n; ++j) {
        double s = 0.0;
        for (int k = 0; k <= n; ++k) {
            double xk = cos(M_PI * (k + 0.5) / (n + 1));
            s += log(1.0 - ((1.0 - 2.0 * delta) * xk + 1.0) / 2.0) * cheb_T(j, xk);
        }
        c[j] = (j == 0 ? 1.0 : 2.0) / (n + 1) * s;
    }
}

/* ------------------------------------------------------------------------- */
/* Matrix-vector products.  CSR with int64 row pointers and int32 columns;    */
/* each row's FP64 sum runs over the stored entries in storage order.         */
/* ------------------------------------------------------------------------- */
static void csr_matvec(int64_t d, const int64_t* rowptr, const int32_t* col,
                       const double* val, const double* x, double* y) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < d; ++i) {
        double s = 0.0;
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) s += val[k] * x[col[k]];
        y[i] = s;
    }
}

/* y = C^T x, as a plain scatter over the rows of C (sequential: no races). */
static void csr_matvec_transpose(int64_t d, const int64_t* rowptr, const int32_t* col,
                                 const double* val, const double* x, double* y) {
    for (int64_t i = 0; i < d; ++i) y[i] = 0.0;
    for (int64_t i = 0; i < d; ++i)
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) y[col[k]] += val[k] * x[i];
}

/* The operator whose log-determinant is estimated.  kind 0: B itself (symmetric
 * positive definite).  kind 1: C^T C applied as C then C^T, never formed
 * (Algorithm 2 and the remark on its O(mn||C||_0) cost, Sec. 3.2). */
typedef struct {
    int kind;
    int64_t d;
    const int64_t* rowptr;
    const int32_t* col;
    const double* val;
    double* tmp; /* d doubles, kind 1 only */
} op_t;

static void op_apply(const op_t* op, const double* x, double* y) {
    if (op->kind == 0) {
        csr_matvec(op->d, op->rowptr, op->col, op->val, x, y);
    } else {
        csr_matvec(op->d, op->rowptr, op->col, op->val, x, op->tmp);
        csr_matvec_transpose(op->d, op->rowptr, op->col, op->val, op->tmp, y);
    }
}

static double dot(int64_t d, const double* x, const double* y) {
    double s = 0.0;
    for (int64_t i = 0; i < d; ++i) s += x[i] * y[i];
    return s;
}

/* ------------------------------------------------------------------------- */
/* Estimator moments, spectral-interval form.                                  */
/*                                                                             */
/* With the spectrum of the operator X (B, or C^T C) inside [a,b], the shifted */
/* matrix At = (2X - (a+b) I) / (b - a) has its spectrum in [-1,1] (the affine */
/* map of Sec. 4.1).  For each probe v (a column of V):                        */
/*   w_0 = v,  w_1 = At v,  w_{j+1} = 2 At w_j - w_{j-1}   (Sec. 2.2)          */
/*   t_j = v^T w_j = v^T T_j(At) v,   j = 0..n.                                */
/* The log-determinant estimate is Gamma = (1/M) sum_p sum_j c_j t_{j,p}       */
/* (Algorithm 1: u = sum_j c_j w_j, Gamma += v^T u / m), and                   */
/* Gamma_p = sum_j c_j t_{j,p} is the per-probe estimate.                      */
/*                                                                             */
/* V: d x M row-major (probe fastest), any real entries (Rademacher for the    */
/* estimator; basis vectors for an exact trace).  t: (n+1) x M row-major.      */
/* Returns 0 on success, -1 on a bad argument, -2 on allocation failure.       */
/* ------------------------------------------------------------------------- */
static int moments_op(const op_t* op, double a, double b, int n, int64_t M,
                      const double* V, double* t) {
    int64_t d = op->d;
    if (d < 0 || n < 0 || M < 0 || !(a < b)) return -1;
    double* v = (double*)malloc(sizeof(double) * (size_t)(d > 0 ? d : 1));
    double* wm = (double*)malloc(sizeof(double) * (size_t)(d > 0 ? d : 1));
    double* w = (double*)malloc(sizeof(double) * (size_t)(d > 0 ? d : 1));
    double* wp = (double*)malloc(sizeof(double) * (size_t)(d > 0 ? d : 1));
    double* bx = (double*)malloc(sizeof(double) * (size_t)(d > 0 ? d : 1));
    if (!v || !wm || !w || !wp || !bx) {
        free(v); free(wm); free(w); free(wp); free(bx);
        return -2;
    }
    const double scale = 2.0 / (b - a), shift = (a + b) / (b - a);
    for (int64_t p = 0; p < M; ++p) {
        for (int64_t i = 0; i < d; ++i) v[i] = V[i * M + p];
        /* w_0 = v */
        memcpy(wm, v, sizeof(double) * (size_t)d);
        t[0 * M + p] = dot(d, v, wm);
        if (n == 0) continue;
        /* w_1 = At v */
        op_apply(op, wm, bx);
        for (int64_t i = 0; i < d; ++i) w[i] = scale * bx[i] - shift * wm[i];
        t[1 * M + p] = dot(d, v, w);
        /* w_{j+1} = 2 At w_j - w_{j-1} */
        for (int j = 1; j < n; ++j) {
            op_apply(op, w, bx);
            for (int64_t i = 0; i < d; ++i) wp[i] = 2.0 * (scale * bx[i] - shift * w[i]) - wm[i];
            t[(int64_t)(j + 1) * M + p] = dot(d, v, wp);
            double* r = wm; wm = w; w = wp; wp = r;
        }
    }
    free(v); free(wm); free(w); free(wp); free(bx);
    return 0;
}

EXPORT int oracle_moments(int64_t d, const int64_t* rowptr, const int32_t* col,
                          const double* val, int kind, double a, double b, int n,
                          int64_t M, const double* V, double* t) {
    op_t op = {kind, d, rowptr, col, val, NULL};
    if (kind == 1) {
        op.tmp = (double*)malloc(sizeof(double) * (size_t)(d > 0 ? d : 1));
        if (!op.tmp) return -2;
    }
    int rc = moments_op(&op, a, b, n, M, V, t);
    free(op.tmp);
    return rc;
}

/* Gamma_p = sum_j c_j t_{j,p};  Gamma = (1/M) sum_p Gamma_p  (Algorithm 1).
 * For kind 1 the result estimates logdet(C^T C) = 2 log|det C| (Algorithm 2);
 * the caller halves it. */
EXPORT void oracle_finalize(int n, int64_t M, const double* c, const double* t,
                            double* gamma_p, double* gamma) {
    double s = 0.0;
    for (int64_t p = 0; p < M; ++p) {
        double g = 0.0;
        for (int j = 0; j <= n; ++j) g += c[j] * t[(int64_t)j * M + p];
        gamma_p[p] = g;
        s += g;
    }
    *gamma = M > 0 ? s / (double)M : 0.0;
}

/* ------------------------------------------------------------------------- */
/* Algorithm 1, literal form.  Input B with eigenvalues in [delta, 1-delta].   */
/* A = I - B; c_i are the coefficients of log(1 - ((1-2 delta) x + 1)/2); for  */
/* each probe u = c_0 v + c_1 w_1 + sum_{j>=2} c_j w_j and Gamma += v^T u / m. */
/* Reading: the polynomial's variable x lives on [-1,1] and is tied to the     */
/* eigenvalue lambda of A by lambda = g(x) = ((1-2 delta) x + 1)/2 (Sec. 4.1), */
/* so the recurrence runs on X = g^{-1}(A) = (2A - I)/(1 - 2 delta); the      */
/* line "IF n > 1" is read as "IF n >= 1" so that n = 1 keeps its c_1 term.    */
/* ------------------------------------------------------------------------- */
static int alg1_literal_op(const op_t* op, double delta, int n, int64_t m,
                           const double* V, double* gamma_out) {
    int64_t d = op->d;
    if (!(delta > 0.0 && delta < 0.5) || n < 0 || m <= 0) return -1;
    double* c = (double*)malloc(sizeof(double) * (size_t)(n + 1));
    double* v = (double*)malloc(sizeof(double) * (size_t)(d > 0 ? d : 1));
    double* u = (double*)malloc(sizeof(double) * (size_t)(d > 0 ? d : 1));
    double* w0 = (double*)malloc(sizeof(double) * (size_t)(d > 0 ? d : 1));
    double* w1 = (double*)malloc(sizeof(double) * (size_t)(d > 0 ? d : 1));
    double* w2 = (double*)malloc(sizeof(double) * (size_t)(d > 0 ? d : 1));
    double* bx = (double*)malloc(sizeof(double) * (size_t)(d > 0 ? d : 1));
    if (!c || !v || !u || !w0 || !w1 || !w2 || !bx) {
        free(c); free(v); free(u); free(w0); free(w1); free(w2); free(bx);
        return -2;
    }
    oracle_cheb_coeffs_alg1(n, delta, c);
    /* X y = (2 (I - B) y - y) / (1 - 2 delta) = (y - 2 B y) / (1 - 2 delta) */
    const double inv = 1.0 / (1.0 - 2.0 * delta);
    double gamma = 0.0;
    for (int64_t p = 0; p < m; ++p) {
        for (int64_t i = 0; i < d; ++i) v[i] = V[i * m + p];
        for (int64_t i = 0; i < d; ++i) u[i] = c[0] * v[i];
        if (n >= 1) {
            memcpy(w0, v, sizeof(double) * (size_t)d);
            op_apply(op, v, bx);
            for (int64_t i = 0; i < d; ++i) w1[i] = (v[i] - 2.0 * bx[i]) * inv;
            for (int64_t i = 0; i < d; ++i) u[i] += c[1] * w1[i];
            for (int j = 2; j <= n; ++j) {
                op_apply(op, w1, bx);
                for (int64_t i = 0; i < d; ++i) w2[i] = 2.0 * ((w1[i] - 2.0 * bx[i]) * inv) - w0[i];
                for (int64_t i = 0; i < d; ++i) u[i] += c[j] * w2[i];
                double* r = w0; w0 = w1; w1 = w2; w2 = r;
            }
        }
        gamma += dot(d, v, u) / (double)m;
    }
    *gamma_out = gamma;
    free(c); free(v); free(u); free(w0); free(w1); free(w2); free(bx);
    return 0;
}

EXPORT int oracle_alg1_literal(int64_t d, const int64_t* rowptr, const int32_t* col,
                               const double* val, double delta, int n, int64_t m,
                               const double* V, double* gamma) {
    op_t op = {0, d, rowptr, col, val, NULL};
    return alg1_literal_op(&op, delta, n, m, V, gamma);
}

/* Algorithm 2: B = C^T C / s with s = sigma_min^2 + sigma_max^2 (applied as C
 * then C^T, scaled), delta = sigma_min^2 / s, Gamma from Algorithm 1, output
 * (Gamma + d log s) / 2, an estimate of log|det C|. */
typedef struct {
    op_t inner;
    double s;
} scaled_op_t;

EXPORT int oracle_alg2_literal(int64_t d, const int64_t* rowptr, const int32_t* col,
                               const double* val, double sigma_min, double sigma_max, int n,
                               int64_t m, const double* V, double* out) {
    double s = sigma_min * sigma_min + sigma_max * sigma_max;
    double delta = sigma_min * sigma_min / s;
    /* Scale the stored values by 1/sqrt(s) so that (C/sqrt s)^T (C/sqrt s) = B. */
    int64_t nnz = rowptr[d];
    double* sval = (double*)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
    double* tmp = (double*)malloc(sizeof(double) * (size_t)(d > 0 ? d : 1));
    if (!sval || !tmp) { free(sval); free(tmp); return -2; }
    double r = 1.0 / sqrt(s);
    for (int64_t k = 0; k < nnz; ++k) sval[k] = val[k] * r;
    op_t op = {1, d, rowptr, col, sval, tmp};
    double gamma = 0.0;
    int rc = alg1_literal_op(&op, delta, n, m, V, &gamma);
    *out = (gamma + (double)d * log(s)) / 2.0;
    free(sval); free(tmp);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Spectral bounds (Sec. 3.2).                                                 */
/* Gershgorin: every eigenvalue of symmetric B lies in                         */
/*   [min_i (B_ii - R_i), max_i (B_ii + R_i)],  R_i = sum_{k != i} |B_ik|.     */
/* Norm bound: sigma_max(C) <= sqrt(||C||_1 ||C||_inf).                        */
/* ------------------------------------------------------------------------- */
EXPORT void oracle_gershgorin(int64_t d, const int64_t* rowptr, const int32_t* col,
                              const double* val, double* lo, double* hi) {
    double l = INFINITY, h = -INFINITY;
    for (int64_t i = 0; i < d; ++i) {
        double diag = 0.0, r = 0.0;
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            if (col[k] == i) diag += val[k];
            else r += fabs(val[k]);
        }
        if (diag - r < l) l = diag - r;
        if (diag + r > h) h = diag + r;
    }
    *lo = l;
    *hi = h;
}

EXPORT double oracle_sigma_max_bound(int64_t d, const int64_t* rowptr, const int32_t* col,
                                     const double* val) {
    double* colsum = (double*)calloc((size_t)(d > 0 ? d : 1), sizeof(double));
    if (!colsum) return NAN;
    double norm_inf = 0.0;
    for (int64_t i = 0; i < d; ++i) {
        double r = 0.0;
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            r += fabs(val[k]);
            colsum[col[k]] += fabs(val[k]);
        }
        if (r > norm_inf) norm_inf = r;
    }
    double norm_1 = 0.0;
    for (int64_t i = 0; i < d; ++i)
        if (colsum[i] > norm_1) norm_1 = colsum[i];
    free(colsum);
    return sqrt(norm_1 * norm_inf);
}

/* Diagonal-dominance margins of a general C (Sec. 3.2: sigma_min is easy for
 * diagonally dominant matrices).  alpha = min_i (|C_ii| - R_i) over rows,
 * beta = min_i (|C_ii| - S_i) over columns (R_i, S_i: off-diagonal absolute
 * row / column sums).  Varah's bounds ||C^-1||_inf <= 1/alpha and
 * ||C^-1||_1 <= 1/beta give sigma_min(C)^2 >= alpha * beta when both are > 0. */
EXPORT void oracle_dominance_margins(int64_t d, const int64_t* rowptr, const int32_t* col,
                                     const double* val, double* alpha, double* beta) {
    double* diag = (double*)calloc((size_t)(d > 0 ? d : 1), sizeof(double));
    double* colsum = (double*)calloc((size_t)(d > 0 ? d : 1), sizeof(double));
    if (!diag || !colsum) { free(diag); free(colsum); *alpha = *beta = NAN; return; }
    double amin = INFINITY;
    for (int64_t i = 0; i < d; ++i) {
        double r = 0.0;
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            if (col[k] == i) diag[i] += val[k];
            else { r += fabs(val[k]); colsum[col[k]] += fabs(val[k]); }
        }
        (void)r;
    }
    for (int64_t i = 0; i < d; ++i) {
        double r = 0.0;
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
            if (col[k] != i) r += fabs(val[k]);
        if (fabs(diag[i]) - r < amin) amin = fabs(diag[i]) - r;
    }
    double bmin = INFINITY;
    for (int64_t i = 0; i < d; ++i)
        if (fabs(diag[i]) - colsum[i] < bmin) bmin = fabs(diag[i]) - colsum[i];
    *alpha = amin;
    *beta = bmin;
    free(diag);
    free(colsum);
}

/* ------------------------------------------------------------------------- */
/* Exact reference: dense Cholesky B = L L^T, log det B = 2 sum_i log L_ii     */
/* (Sec. 1).  A is d x d row-major and is overwritten by L in its lower part. */
/* Returns 0, or -1 if a pivot is not positive (B not positive definite).     */
/* ------------------------------------------------------------------------- */
EXPORT int oracle_logdet_cholesky(int64_t d, double* A, double* logdet) {
    double s = 0.0;
    for (int64_t j = 0; j < d; ++j) {
        double piv = A[j * d + j];
        for (int64_t k = 0; k < j; ++k) piv -= A[j * d + k] * A[j * d + k];
        if (!(piv > 0.0)) return -1;
        double ljj = sqrt(piv);
        A[j * d + j] = ljj;
        s += log(ljj);
#pragma omp parallel for schedule(static)
        for (int64_t i = j + 1; i < d; ++i) {
            double x = A[i * d + j];
            for (int64_t k = 0; k < j; ++k) x -= A[i * d + k] * A[j * d + k];
            A[i * d + j] = x / ljj;
        }
    }
    *logdet = 2.0 * s;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Gradient of the estimate with respect to the stored values (extension).     */
/*                                                                             */
/* Gamma = (1/M) sum_p sum_{j=0..n} c_j v_p^T T_j(At) v_p with                 */
/* At = (2B - (a+b)I)/(b-a), the interval [a,b] held fixed.  For symmetric B   */
/* and an entry perturbation dB, with w_i = T_i(At) v, the chain rule through   */
/* the recurrence, one degree at a time, reads                                  */
/*   dw_0 = 0, dw_1 = dAt v, dw_{i+1} = 2 dAt w_i + 2 At dw_i - dw_{i-1},      */
/* so d t_j = v^T dw_j.  Rather than propagate dw for every entry, the adjoint */
/* vectors are formed by the same recurrence run backwards:                    */
/*   lambda_{n+1} = lambda_{n+2} = 0,                                          */
/*   lambda_i = c_i v + 2 At lambda_{i+1} - lambda_{i+2}   (i = n..1),         */
/* and dGamma_p = lambda_1^T dAt v + 2 sum_{i=1}^{n-1} lambda_{i+1}^T dAt w_i.  */
/* With dAt = (2/(b-a)) dB, the derivative with respect to a stored entry      */
/* (r, k) (treated as an independent value, no symmetry tie) is               */
/*   G_rk = (2/(b-a)) [ lambda_1[r] v[k] + 2 sum_{i=1}^{n-1} lambda_{i+1}[r] w_i[k] ]. */
/* The result is averaged over probes.  The derivation is checked against     */
/* finite differences of oracle_moments + oracle_finalize and, for its mean,  */
/* against tr(B^{-1} dB) from the dense Cholesky reference.                  */
/* G: nnz doubles (output).                                                    */
/* ------------------------------------------------------------------------- */
EXPORT int oracle_grad(int64_t d, const int64_t* rowptr, const int32_t* col,
                       const double* val, double a, double b, int n, int64_t M,
                       const double* V, double* G) {
    if (d < 0 || n < 0 || M <= 0 || !(a < b)) return -1;
    int64_t nnz = rowptr[d];
    for (int64_t k = 0; k < nnz; ++k) G[k] = 0.0;
    if (n == 0 || d == 0) return 0;
    const double scale = 2.0 / (b - a), shift = (a + b) / (b - a);
    double* c = (double*)malloc(sizeof(double) * (size_t)(n + 1));
    double* v = (double*)malloc(sizeof(double) * (size_t)d);
    double* W = (double*)malloc(sizeof(double) * (size_t)d * (size_t)(n + 1)); /* w_0..w_n */
    double* L = (double*)malloc(sizeof(double) * (size_t)d * (size_t)(n + 3)); /* lambda_0..lambda_{n+2} */
    double* bx = (double*)malloc(sizeof(double) * (size_t)d);
    if (!c || !v || !W || !L || !bx) {
        free(c); free(v); free(W); free(L); free(bx);
        return -2;
    }
    oracle_cheb_coeffs(n, a, b, c);
    op_t op = {0, d, rowptr, col, val, NULL};
    for (int64_t p = 0; p < M; ++p) {
        for (int64_t i = 0; i < d; ++i) v[i] = V[i * M + p];
        /* forward: store every w_i */
        double* w0 = W;
        memcpy(w0, v, sizeof(double) * (size_t)d);
        if (n >= 1) {
            double* w1 = W + d;
            op_apply(&op, w0, bx);
            for (int64_t i = 0; i < d; ++i) w1[i] = scale * bx[i] - shift * w0[i];
        }
        for (int j = 1; j < n; ++j) {
            double* wj = W + (int64_t)j * d;
            double* wjm = W + (int64_t)(j - 1) * d;
            double* wjp = W + (int64_t)(j + 1) * d;
            op_apply(&op, wj, bx);
            for (int64_t i = 0; i < d; ++i) wjp[i] = 2.0 * (scale * bx[i] - shift * wj[i]) - wjm[i];
        }
        /* backward: lambda_i = c_i v + 2 At lambda_{i+1} - lambda_{i+2}, i = n..1 */
        for (int64_t i = 0; i < d; ++i) {
            L[(int64_t)(n + 1) * d + i] = 0.0;
            L[(int64_t)(n + 2) * d + i] = 0.0;
        }
        for (int j = n; j >= 1; --j) {
            double* lj = L + (int64_t)j * d;
            double* l1 = L + (int64_t)(j + 1) * d;
            double* l2 = L + (int64_t)(j + 2) * d;
            op_apply(&op, l1, bx);
            for (int64_t i = 0; i < d; ++i)
                lj[i] = c[j] * v[i] + 2.0 * (scale * bx[i] - shift * l1[i]) - l2[i];
        }
        /* accumulate G_rk over the stored entries */
#pragma omp parallel for schedule(static)
        for (int64_t r = 0; r < d; ++r) {
            for (int64_t k = rowptr[r]; k < rowptr[r + 1]; ++k) {
                int64_t cc = col[k];
                double g = L[1 * d + r] * v[cc];
                for (int i = 1; i <= n - 1; ++i) g += 2.0 * L[(int64_t)(i + 1) * d + r] * W[(int64_t)i * d + cc];
                G[k] += scale * g / (double)M;
            }
        }
    }
    free(c); free(v); free(W); free(L); free(bx);
    return 0;
}

EXPORT int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
