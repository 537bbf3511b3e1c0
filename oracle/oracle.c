/*
 * oracle.c -- plain, slow, obviously correct CPU reference for the
 * mixed-precision iterative-refinement solver.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The product path
 * (the CUDA library) shares no code, header or constant with it.
 *
 * Source: Baboulin, Buttari, Dongarra, Kurzak, Langou, Langou, Luszczek,
 * Tomov, "Accelerating Scientific Computations with Mixed Precision
 * Algorithms".  Every routine names the passage it follows.
 *
 * Conventions: all matrices are column-major with a leading dimension;
 * pivots are LAPACK style (1-based, row i was exchanged with row ipiv[i],
 * applied in increasing i).  Arithmetic is FP64 unless the routine name
 * says FP32 (the paper fixes single precision for the factorization and the
 * triangular solves of Algorithm 1, Section 2.1).
 *
 * No blocking, no reordering: loops run in the textbook order so that a
 * reader can check them against the paper.  OpenMP is used only across the
 * independent columns of a rank-1 update and across independent rows of a
 * residual, which leaves the per-element operation order (and therefore
 * every result bit) independent of the thread count.
 *
 * Parity status per routine (pins live in the tests):
 *   getrf/getrs/potrf/potrs (FP64, FP32) : pinned (exact rationals, closed forms)
 *   getrs_trans                         : pinned (exact rational solve of A^T x = b
 *                                         on matrices that must pivot)
 *   residual, residual_dot2, matvec_dot2 : pinned (exact rationals, cancelling sums)
 *   norm_inf, bwd_err                   : pinned (exact rationals)
 *   gesv_ir, posv_ir                    : pinned (special cases, closed forms,
 *                                         Datta iteration-count prediction)
 *   kappa_inf_exact, kappa_1_est,       : pinned (Hilbert / tridiagonal closed forms;
 *   dinvnorm1_est_lu                      lower bound within 10x of the exact norm)
 *   gmres_ir                            : pinned (special cases, exact solve bound)
 *   gesv_dd                             : pinned (exact rational solves, including a
 *                                         floating-point Hilbert matrix, kappa ~ 1e13)
 *   round_bf16/fp16/e4m3                : pinned (enumerated representable values)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define IDX(i, j, ld) ((size_t)(j) * (size_t)(ld) + (size_t)(i))

/* ------------------------------------------------------------------ */
/* Thread control (the timed CPU baseline reports its thread count).   */
/* ------------------------------------------------------------------ */
int or_set_threads(int nt) {
#ifdef _OPENMP
    if (nt > 0) omp_set_num_threads(nt);
    return omp_get_max_threads();
#else
    (void)nt;
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* LU with partial pivoting, PA = LU  (Section 2.1, first paragraph;   */
/* Algorithm 1 step 1).  Unblocked right-looking Gaussian elimination:  */
/* pivot = largest magnitude in the column (ties: smallest row index),  */
/* swap whole rows, scale by division, rank-1 update.  A zero pivot     */
/* records info = k+1 (first one) and the elimination continues, as in  */
/* LAPACK xGETF2 which the paper's SGETRF/DGETRF build on (Section 3.1.1).*/
/* ------------------------------------------------------------------ */
int or_dgetrf(int n, double *A, int lda, int *ipiv) {
    int info = 0;
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = fabs(A[IDX(k, k, lda)]);
        for (int i = k + 1; i < n; ++i) {
            double v = fabs(A[IDX(i, k, lda)]);
            if (v > best) { best = v; p = i; }
        }
        ipiv[k] = p + 1;
        if (A[IDX(p, k, lda)] == 0.0) {
            if (info == 0) info = k + 1;
            continue;
        }
        if (p != k) {
            for (int j = 0; j < n; ++j) {
                double t = A[IDX(k, j, lda)];
                A[IDX(k, j, lda)] = A[IDX(p, j, lda)];
                A[IDX(p, j, lda)] = t;
            }
        }
        double piv = A[IDX(k, k, lda)];
        for (int i = k + 1; i < n; ++i) A[IDX(i, k, lda)] /= piv;
#pragma omp parallel for schedule(static) if (n - k > 256)
        for (int j = k + 1; j < n; ++j) {
            double ukj = A[IDX(k, j, lda)];
            if (ukj == 0.0) continue;
            double *colj = &A[IDX(0, j, lda)];
            const double *colk = &A[IDX(0, k, lda)];
            for (int i = k + 1; i < n; ++i) colj[i] -= colk[i] * ukj;
        }
    }
    return info;
}

/* Same elimination entirely in IEEE single precision: step 1 of
 * Algorithm 1 at precision eps_s (Section 2.1; SGETRF, Section 3.1.1). */
int or_sgetrf(int n, float *A, int lda, int *ipiv) {
    int info = 0;
    for (int k = 0; k < n; ++k) {
        int p = k;
        float best = fabsf(A[IDX(k, k, lda)]);
        for (int i = k + 1; i < n; ++i) {
            float v = fabsf(A[IDX(i, k, lda)]);
            if (v > best) { best = v; p = i; }
        }
        ipiv[k] = p + 1;
        if (A[IDX(p, k, lda)] == 0.0f) {
            if (info == 0) info = k + 1;
            continue;
        }
        if (p != k) {
            for (int j = 0; j < n; ++j) {
                float t = A[IDX(k, j, lda)];
                A[IDX(k, j, lda)] = A[IDX(p, j, lda)];
                A[IDX(p, j, lda)] = t;
            }
        }
        float piv = A[IDX(k, k, lda)];
        for (int i = k + 1; i < n; ++i) A[IDX(i, k, lda)] /= piv;
#pragma omp parallel for schedule(static) if (n - k > 256)
        for (int j = k + 1; j < n; ++j) {
            float ukj = A[IDX(k, j, lda)];
            if (ukj == 0.0f) continue;
            float *colj = &A[IDX(0, j, lda)];
            const float *colk = &A[IDX(0, k, lda)];
            for (int i = k + 1; i < n; ++i) colj[i] = colj[i] - colk[i] * ukj;
        }
    }
    return info;
}

/* Forward then backward substitution with the LU factors: Ly = Pb,
 * Ux = y (Section 2.1; Algorithm 1 steps 2-3 and 5-6).  B is overwritten
 * by X.  Rows are visited in order 0..n-1 (forward) and n-1..0 (back). */
void or_dgetrs(int n, int nrhs, const double *LU, int lda, const int *ipiv,
               double *B, int ldb) {
    for (int c = 0; c < nrhs; ++c) {
        double *b = &B[IDX(0, c, ldb)];
        for (int k = 0; k < n; ++k) {
            int p = ipiv[k] - 1;
            if (p != k) { double t = b[k]; b[k] = b[p]; b[p] = t; }
        }
        for (int i = 0; i < n; ++i) {
            double s = b[i];
            for (int j = 0; j < i; ++j) s -= LU[IDX(i, j, lda)] * b[j];
            b[i] = s;
        }
        for (int i = n - 1; i >= 0; --i) {
            double s = b[i];
            for (int j = i + 1; j < n; ++j) s -= LU[IDX(i, j, lda)] * b[j];
            b[i] = s / LU[IDX(i, i, lda)];
        }
    }
}

void or_sgetrs(int n, int nrhs, const float *LU, int lda, const int *ipiv,
               float *B, int ldb) {
    for (int c = 0; c < nrhs; ++c) {
        float *b = &B[IDX(0, c, ldb)];
        for (int k = 0; k < n; ++k) {
            int p = ipiv[k] - 1;
            if (p != k) { float t = b[k]; b[k] = b[p]; b[p] = t; }
        }
        for (int i = 0; i < n; ++i) {
            float s = b[i];
            for (int j = 0; j < i; ++j) s = s - LU[IDX(i, j, lda)] * b[j];
            b[i] = s;
        }
        for (int i = n - 1; i >= 0; --i) {
            float s = b[i];
            for (int j = i + 1; j < n; ++j) s = s - LU[IDX(i, j, lda)] * b[j];
            b[i] = s / LU[IDX(i, i, lda)];
        }
    }
}

/* Transposed solve with the same factors: A^T x = b  <=>  U^T L^T P x = b.
 * Used for the adjoint of the solve (gradient of x = A^{-1} b). */
void or_dgetrs_trans(int n, int nrhs, const double *LU, int lda,
                     const int *ipiv, double *B, int ldb) {
    for (int c = 0; c < nrhs; ++c) {
        double *b = &B[IDX(0, c, ldb)];
        for (int i = 0; i < n; ++i) {            /* U^T w = b */
            double s = b[i];
            for (int j = 0; j < i; ++j) s -= LU[IDX(j, i, lda)] * b[j];
            b[i] = s / LU[IDX(i, i, lda)];
        }
        for (int i = n - 1; i >= 0; --i) {       /* L^T v = w */
            double s = b[i];
            for (int j = i + 1; j < n; ++j) s -= LU[IDX(j, i, lda)] * b[j];
            b[i] = s;
        }
        for (int k = n - 1; k >= 0; --k) {       /* x = P^T v */
            int p = ipiv[k] - 1;
            if (p != k) { double t = b[k]; b[k] = b[p]; b[p] = t; }
        }
    }
}

/* ------------------------------------------------------------------ */
/* Cholesky A = L L^T, lower (Section 3.1.1: SPOTRF for the symmetric   */
/* case; Section 6).  Left-looking plain loops.  A non-positive (or     */
/* non-finite) pivot returns info = k+1 and stops.                      */
/* ------------------------------------------------------------------ */
int or_dpotrf(int n, double *A, int lda) {
    for (int k = 0; k < n; ++k) {
        double d = A[IDX(k, k, lda)];
        for (int j = 0; j < k; ++j) d -= A[IDX(k, j, lda)] * A[IDX(k, j, lda)];
        if (!(d > 0.0) || !isfinite(d)) return k + 1;
        double lkk = sqrt(d);
        A[IDX(k, k, lda)] = lkk;
#pragma omp parallel for schedule(static) if (n - k > 256)
        for (int i = k + 1; i < n; ++i) {
            double s = A[IDX(i, k, lda)];
            for (int j = 0; j < k; ++j) s -= A[IDX(i, j, lda)] * A[IDX(k, j, lda)];
            A[IDX(i, k, lda)] = s / lkk;
        }
    }
    return 0;
}

int or_spotrf(int n, float *A, int lda) {
    for (int k = 0; k < n; ++k) {
        float d = A[IDX(k, k, lda)];
        for (int j = 0; j < k; ++j) d = d - A[IDX(k, j, lda)] * A[IDX(k, j, lda)];
        if (!(d > 0.0f) || !isfinite(d)) return k + 1;
        float lkk = sqrtf(d);
        A[IDX(k, k, lda)] = lkk;
#pragma omp parallel for schedule(static) if (n - k > 256)
        for (int i = k + 1; i < n; ++i) {
            float s = A[IDX(i, k, lda)];
            for (int j = 0; j < k; ++j) s = s - A[IDX(i, j, lda)] * A[IDX(k, j, lda)];
            A[IDX(i, k, lda)] = s / lkk;
        }
    }
    return 0;
}

/* L y = b, then L^T x = y (SPOTRS / DPOTRS, Section 3.1.1). */
void or_dpotrs(int n, int nrhs, const double *L, int lda, double *B, int ldb) {
    for (int c = 0; c < nrhs; ++c) {
        double *b = &B[IDX(0, c, ldb)];
        for (int i = 0; i < n; ++i) {
            double s = b[i];
            for (int j = 0; j < i; ++j) s -= L[IDX(i, j, lda)] * b[j];
            b[i] = s / L[IDX(i, i, lda)];
        }
        for (int i = n - 1; i >= 0; --i) {
            double s = b[i];
            for (int j = i + 1; j < n; ++j) s -= L[IDX(j, i, lda)] * b[j];
            b[i] = s / L[IDX(i, i, lda)];
        }
    }
}

void or_spotrs(int n, int nrhs, const float *L, int lda, float *B, int ldb) {
    for (int c = 0; c < nrhs; ++c) {
        float *b = &B[IDX(0, c, ldb)];
        for (int i = 0; i < n; ++i) {
            float s = b[i];
            for (int j = 0; j < i; ++j) s = s - L[IDX(i, j, lda)] * b[j];
            b[i] = s / L[IDX(i, i, lda)];
        }
        for (int i = n - 1; i >= 0; --i) {
            float s = b[i];
            for (int j = i + 1; j < n; ++j) s = s - L[IDX(j, i, lda)] * b[j];
            b[i] = s / L[IDX(i, i, lda)];
        }
    }
}

/* ------------------------------------------------------------------ */
/* Residual r = b - A x in FP64 (Algorithm 1 step 4, eps_d; DGEMM in    */
/* Section 3.1.1).  Each row accumulates over columns j = 0..n-1 in     */
/* order, starting from b.                                              */
/* ------------------------------------------------------------------ */
void or_dresidual(int n, int nrhs, const double *A, int lda, const double *X,
                  int ldx, const double *B, int ldb, double *R, int ldr) {
    for (int c = 0; c < nrhs; ++c) {
        const double *x = &X[IDX(0, c, ldx)];
        double *r = &R[IDX(0, c, ldr)];
        const double *b = &B[IDX(0, c, ldb)];
#pragma omp parallel for schedule(static) if (n > 512)
        for (int i = 0; i < n; ++i) {
            double s = b[i];
            for (int j = 0; j < n; ++j) s -= A[IDX(i, j, lda)] * x[j];
            r[i] = s;
        }
    }
}

/* Error-free transformations (Knuth TwoSum; TwoProduct via fused
 * multiply-add) and the compensated dot product Dot2 of Ogita, Rump and
 * Oishi (2005).  The checker's residual is then as accurate as if it had
 * been computed in twice the working precision and rounded once, so the
 * backward error it reports does not depend on either side's summation
 * order.  The paper leaves the stopping test open (Section 2.1, last
 * paragraph); this is the measuring instrument, not the method. */
static inline void two_sum(double a, double b, double *s, double *e) {
    double x = a + b;
    double z = x - a;
    *e = (a - (x - z)) + (b - z);
    *s = x;
}
static inline void two_prod(double a, double b, double *p, double *e) {
    double x = a * b;
    *e = fma(a, b, -x);
    *p = x;
}

void or_dresidual_dot2(int n, int nrhs, const double *A, int lda,
                       const double *X, int ldx, const double *B, int ldb,
                       double *R, int ldr) {
    for (int c = 0; c < nrhs; ++c) {
        const double *x = &X[IDX(0, c, ldx)];
        double *r = &R[IDX(0, c, ldr)];
        const double *b = &B[IDX(0, c, ldb)];
#pragma omp parallel for schedule(static) if (n > 512)
        for (int i = 0; i < n; ++i) {
            double s = b[i], comp = 0.0;
            for (int j = 0; j < n; ++j) {
                double p, ep, t, es;
                two_prod(-A[IDX(i, j, lda)], x[j], &p, &ep);
                two_sum(s, p, &t, &es);
                s = t;
                comp += ep + es;
            }
            r[i] = s + comp;
        }
    }
}

/* Compensated product b = A x (same Dot2), used to form right-hand sides
 * that are accurate to one rounding. */
void or_dmatvec_dot2(int n, int nrhs, const double *A, int lda,
                     const double *X, int ldx, double *B, int ldb) {
    for (int c = 0; c < nrhs; ++c) {
        const double *x = &X[IDX(0, c, ldx)];
        double *b = &B[IDX(0, c, ldb)];
#pragma omp parallel for schedule(static) if (n > 512)
        for (int i = 0; i < n; ++i) {
            double s = 0.0, comp = 0.0;
            for (int j = 0; j < n; ++j) {
                double p, ep, t, es;
                two_prod(A[IDX(i, j, lda)], x[j], &p, &ep);
                two_sum(s, p, &t, &es);
                s = t;
                comp += ep + es;
            }
            b[i] = s + comp;
        }
    }
}

/* ||A||_inf = max_i sum_j |a_ij| (DLANGE, Table 7). */
double or_dnorm_inf(int m, int n, const double *A, int lda) {
    double best = 0.0;
    for (int i = 0; i < m; ++i) {
        double s = 0.0;
        for (int j = 0; j < n; ++j) s += fabs(A[IDX(i, j, lda)]);
        if (s > best || isnan(s)) best = s;
    }
    return best;
}

/* Normwise backward error of each column of X:
 *   bwd_c = ||b_c - A x_c||_inf / (||A||_inf ||x_c||_inf + ||b_c||_inf),
 * the infinity-norm form of the accuracy test of Section 3 (the paper
 * states it with 2-norms; the stopping criterion itself is left open in
 * Section 2.1).  The residual is the compensated one. */
void or_bwd_err(int n, int nrhs, const double *A, int lda, const double *X,
                int ldx, const double *B, int ldb, double *bwd) {
    double anorm = or_dnorm_inf(n, n, A, lda);
    double *R = (double *)malloc(sizeof(double) * (size_t)n * (size_t)(nrhs > 0 ? nrhs : 1));
    or_dresidual_dot2(n, nrhs, A, lda, X, ldx, B, ldb, R, n);
    for (int c = 0; c < nrhs; ++c) {
        double rn = 0.0, xn = 0.0, bn = 0.0;
        for (int i = 0; i < n; ++i) {
            double rv = fabs(R[IDX(i, c, n)]);
            double xv = fabs(X[IDX(i, c, ldx)]);
            double bv = fabs(B[IDX(i, c, ldb)]);
            if (rv > rn || isnan(rv)) rn = rv;
            if (xv > xn || isnan(xv)) xn = xv;
            if (bv > bn) bn = bv;
        }
        double den = anorm * xn + bn;
        bwd[c] = (den > 0.0) ? rn / den : (rn > 0.0 ? INFINITY : 0.0);
    }
    free(R);
}

/* ------------------------------------------------------------------ */
/* Mixed-precision iterative refinement, Algorithm 1 (Section 2.1).     */
/*                                                                      */
/*   1: LU <- PA                       (factor precision)               */
/*   2-3: solve Ly = Pb, U x_0 = y     (factor precision)               */
/*   do k = 1, 2, ...                                                   */
/*   4:   r_k <- b - A x_{k-1}         (FP64, original FP64 A)          */
/*        check convergence on x_{k-1}                                   */
/*   5-6: solve L y = P r_k, U z_k = y (factor precision)               */
/*   7:   x_k <- x_{k-1} + z_k         (FP64)                            */
/*                                                                      */
/* factor_prec: 32 = IEEE single (the paper's method), 64 = double      */
/* (classical refinement used to produce the reference solution).       */
/* Convergence test (the paper leaves it open, Section 2.1; Section 3   */
/* stops "as accurate as the full double precision" solve): x_k is      */
/* accepted when, per column, the normwise backward error is <= tol AND */
/* x_k has reached the FP64 floor: bwd == 0, or bwd <= 2 u64 (then     */
/* ||x - x_k|| <= ||A^-1|| ||r|| <= 2 kappa bwd ||x_k||, so the forward */
/* error is at most 4 kappa u64), or the last correction is             */
/* <= 4 u64 ||x_k||, or the corrections stopped shrinking (||z_k|| >     */
/* stall_ratio ||z_{k-1}||, k >= 2).  The same shrink test with bwd >   */
/* tol is a stall (Demmel et al. 2006, cited in Section 2.1).  iter     */
/* counts the corrections applied.  On breakdown, stall or non-convergence the   */
/* routine resorts to the FP64 solve (Section 4: "resort to the         */
/* standard double precision solver") when allow_fallback != 0.         */
/* The low-precision solves scale r by s = 2^ceil(log2 ||r||_inf)       */
/* (exact) before rounding it to single precision and multiply z by s   */
/* after, so that tiny late residuals do not underflow.                 */
/*                                                                      */
/* flags: 1 fallback, 2 stalled, 4 low-precision breakdown,             */
/*        8 non-finite input.  Returns info (>0: FP64 factor singular).  */
/* ------------------------------------------------------------------ */
#define OR_FALLBACK 1u
#define OR_STALLED 2u
#define OR_BREAKDOWN 4u
#define OR_NONFINITE 8u

static double pow2_ceil(double v) {
    if (!(v > 0.0) || !isfinite(v)) return 1.0;
    int e;
    double m = frexp(v, &e); /* v = m * 2^e, m in [0.5, 1) */
    if (m == 0.5) return ldexp(1.0, e - 1);
    return ldexp(1.0, e);
}

static int all_finite(const double *v, size_t len) {
    for (size_t i = 0; i < len; ++i)
        if (!isfinite(v[i])) return 0;
    return 1;
}

int or_gesv_ir(int n, int nrhs, const double *A, int lda, const double *B,
               int ldb, double *X, int ldx, int factor_prec, int itermax,
               double tol, double stall_ratio, int allow_fallback,
               int *iter_out, unsigned *flags_out, double *bwd_out,
               int *hist_len, double *hist) {
    unsigned flags = 0;
    int info = 0, iter = 0;
    size_t nn = (size_t)n * (size_t)n;
    int *ipiv = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    double *R = (double *)malloc(sizeof(double) * (size_t)n * (size_t)(nrhs > 0 ? nrhs : 1));
    double *bwd = (double *)malloc(sizeof(double) * (size_t)(nrhs > 0 ? nrhs : 1));
    double *znorm_prev = (double *)calloc((size_t)(nrhs > 0 ? nrhs : 1), sizeof(double));
    int nh = 0;
    int converged = 0, fail = 0;
    double *zlast = (double *)calloc((size_t)(nrhs > 0 ? nrhs : 1), sizeof(double));

    for (int c = 0; c < nrhs; ++c)
        if (!all_finite(&B[IDX(0, c, ldb)], (size_t)n)) flags |= OR_NONFINITE;
    for (int j = 0; j < n; ++j)
        if (!all_finite(&A[IDX(0, j, lda)], (size_t)n)) flags |= OR_NONFINITE;

    if (factor_prec == 32) {
        float *W = (float *)malloc(sizeof(float) * (nn ? nn : 1));
        float *Z = (float *)malloc(sizeof(float) * (size_t)n * (size_t)(nrhs > 0 ? nrhs : 1));
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) W[IDX(i, j, n)] = (float)A[IDX(i, j, lda)];
        int sinfo = (flags & OR_NONFINITE) ? 1 : or_sgetrf(n, W, n, ipiv);
        if (sinfo != 0) {
            flags |= OR_BREAKDOWN;
            fail = 1;
        }
        for (int j = 0; !fail && j < n; ++j)
            if (!isfinite(W[IDX(j, j, n)])) { flags |= OR_BREAKDOWN; fail = 1; }
        if (!fail) {
            /* steps 2-3: x_0 from b (scaled like every other right-hand side) */
            for (int c = 0; c < nrhs; ++c) {
                double bn = 0.0;
                for (int i = 0; i < n; ++i) bn = fmax(bn, fabs(B[IDX(i, c, ldb)]));
                double s = pow2_ceil(bn);
                for (int i = 0; i < n; ++i) Z[IDX(i, c, n)] = (float)(B[IDX(i, c, ldb)] / s);
                or_sgetrs(n, 1, W, n, ipiv, &Z[IDX(0, c, n)], n);
                for (int i = 0; i < n; ++i) X[IDX(i, c, ldx)] = (double)Z[IDX(i, c, n)] * s;
            }
            double anorm = or_dnorm_inf(n, n, A, lda);
            /* ||z|| of the last and the previous correction; x_0 counts as the
             * first "correction" from zero */
            for (int c = 0; c < nrhs; ++c) {
                double xn = 0.0;
                for (int i = 0; i < n; ++i) xn = fmax(xn, fabs(X[IDX(i, c, ldx)]));
                zlast[c] = xn;
                znorm_prev[c] = 0.0;
            }
            for (;;) {
                /* step 4: r = b - A x (FP64) and the convergence check */
                or_dresidual(n, nrhs, A, lda, X, ldx, B, ldb, R, n);
                double worst = 0.0;
                int done = 1, nonfinite = 0, stalled = 0;
                for (int c = 0; c < nrhs; ++c) {
                    double rn = 0.0, xn = 0.0, bn = 0.0;
                    for (int i = 0; i < n; ++i) {
                        rn = fmax(rn, fabs(R[IDX(i, c, n)]));
                        xn = fmax(xn, fabs(X[IDX(i, c, ldx)]));
                        bn = fmax(bn, fabs(B[IDX(i, c, ldb)]));
                        if (!isfinite(R[IDX(i, c, n)]) || !isfinite(X[IDX(i, c, ldx)])) nonfinite = 1;
                    }
                    double den = anorm * xn + bn;
                    bwd[c] = den > 0.0 ? rn / den : (rn > 0.0 ? INFINITY : 0.0);
                    int stagnant = iter >= 2 && zlast[c] > stall_ratio * znorm_prev[c];
                    int at_floor = bwd[c] == 0.0 || bwd[c] <= 2.0 * 0x1p-53 || zlast[c] <= 4.0 * 0x1p-53 * xn || stagnant;
                    if (!(bwd[c] <= tol && at_floor)) done = 0;
                    if (!(bwd[c] <= tol) && stagnant) stalled = 1;
                    if (bwd[c] > worst || isnan(bwd[c])) worst = bwd[c];
                }
                if (nh < 32) hist[nh++] = worst;
                if (nonfinite) { flags |= OR_BREAKDOWN; fail = 1; break; }
                if (done) { converged = 1; break; }
                if (stalled) { flags |= OR_STALLED; fail = 1; break; }
                if (iter >= itermax) {
                    /* out of corrections: converged only if every column meets tol */
                    int ok = 1;
                    for (int c = 0; c < nrhs; ++c) if (!(bwd[c] <= tol)) ok = 0;
                    if (ok) converged = 1; else fail = 1;
                    break;
                }
                /* steps 5-7 */
                for (int c = 0; c < nrhs; ++c) {
                    double rn = 0.0;
                    for (int i = 0; i < n; ++i) rn = fmax(rn, fabs(R[IDX(i, c, n)]));
                    double s = pow2_ceil(rn);
                    for (int i = 0; i < n; ++i) Z[IDX(i, c, n)] = (float)(R[IDX(i, c, n)] / s);
                    or_sgetrs(n, 1, W, n, ipiv, &Z[IDX(0, c, n)], n);
                    double zn = 0.0;
                    for (int i = 0; i < n; ++i) {
                        double z = (double)Z[IDX(i, c, n)] * s;
                        X[IDX(i, c, ldx)] += z;
                        zn = fmax(zn, fabs(z));
                    }
                    znorm_prev[c] = zlast[c];
                    zlast[c] = zn;
                }
                ++iter;
            }
        }
        free(W);
        free(Z);
    } else {
        /* factor_prec == 64: classical refinement entirely in FP64. */
        double *F = (double *)malloc(sizeof(double) * (nn ? nn : 1));
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) F[IDX(i, j, n)] = A[IDX(i, j, lda)];
        info = or_dgetrf(n, F, n, ipiv);
        if (info == 0) {
            for (int c = 0; c < nrhs; ++c)
                for (int i = 0; i < n; ++i) X[IDX(i, c, ldx)] = B[IDX(i, c, ldb)];
            for (int c = 0; c < nrhs; ++c) or_dgetrs(n, 1, F, n, ipiv, &X[IDX(0, c, ldx)], ldx);
            double anorm = or_dnorm_inf(n, n, A, lda);
            for (int c = 0; c < nrhs; ++c) {
                double xn = 0.0;
                for (int i = 0; i < n; ++i) xn = fmax(xn, fabs(X[IDX(i, c, ldx)]));
                zlast[c] = xn;
                znorm_prev[c] = 0.0;
            }
            for (;;) {
                or_dresidual(n, nrhs, A, lda, X, ldx, B, ldb, R, n);
                int done = 1;
                double worst = 0.0;
                for (int c = 0; c < nrhs; ++c) {
                    double rn = 0.0, xn = 0.0, bn = 0.0;
                    for (int i = 0; i < n; ++i) {
                        rn = fmax(rn, fabs(R[IDX(i, c, n)]));
                        xn = fmax(xn, fabs(X[IDX(i, c, ldx)]));
                        bn = fmax(bn, fabs(B[IDX(i, c, ldb)]));
                    }
                    double den = anorm * xn + bn;
                    bwd[c] = den > 0.0 ? rn / den : (rn > 0.0 ? INFINITY : 0.0);
                    int stagnant = iter >= 2 && zlast[c] > stall_ratio * znorm_prev[c];
                    int at_floor = bwd[c] == 0.0 || bwd[c] <= 2.0 * 0x1p-53 || zlast[c] <= 4.0 * 0x1p-53 * xn || stagnant;
                    if (!(bwd[c] <= tol && at_floor)) done = 0;
                    if (bwd[c] > worst || isnan(bwd[c])) worst = bwd[c];
                }
                if (nh < 32) hist[nh++] = worst;
                if (done || iter >= itermax) break;
                for (int c = 0; c < nrhs; ++c) {
                    or_dgetrs(n, 1, F, n, ipiv, &R[IDX(0, c, n)], n);
                    double zn = 0.0;
                    for (int i = 0; i < n; ++i) {
                        X[IDX(i, c, ldx)] += R[IDX(i, c, n)];
                        zn = fmax(zn, fabs(R[IDX(i, c, n)]));
                    }
                    znorm_prev[c] = zlast[c];
                    zlast[c] = zn;
                }
                ++iter;
            }
        }
        free(F);
    }

    if (factor_prec == 32 && fail && allow_fallback) {
        /* Section 4: resort to the standard double precision solver. */
        int it64 = 0;
        unsigned f64 = 0;
        double bwd64;
        int nh64 = 0;
        double h64[32];
        info = or_gesv_ir(n, nrhs, A, lda, B, ldb, X, ldx, 64, 5, tol, stall_ratio, 0,
                          &it64, &f64, &bwd64, &nh64, h64);
        flags |= OR_FALLBACK;
        iter = -1;
    } else if (factor_prec == 32 && fail) {
        /* no fallback: report the failure, keep the last iterate */
    }
    (void)converged;
    double worst = 0.0;
    or_bwd_err(n, nrhs, A, lda, X, ldx, B, ldb, bwd);
    for (int c = 0; c < nrhs; ++c)
        if (bwd[c] > worst || isnan(bwd[c])) worst = bwd[c];
    *iter_out = iter;
    *flags_out = flags;
    *bwd_out = worst;
    *hist_len = nh;
    free(ipiv);
    free(R);
    free(bwd);
    free(znorm_prev);
    free(zlast);
    return info;
}

/* Algorithm 1 for SPD A with a Cholesky factorization (SPOTRF, SPOTRS,
 * DSYMM: Section 3.1.1; Section 6).  Same control flow as or_gesv_ir; the
 * FP64 residual uses the full symmetric A (the result is the same as
 * reading one triangle, up to summation order).  A non-positive pivot in
 * single precision is a breakdown. */
int or_posv_ir(int n, int nrhs, const double *A, int lda, const double *B,
               int ldb, double *X, int ldx, int factor_prec, int itermax,
               double tol, double stall_ratio, int allow_fallback,
               int *iter_out, unsigned *flags_out, double *bwd_out) {
    unsigned flags = 0;
    int info = 0, iter = 0, fail = 0;
    size_t nn = (size_t)n * (size_t)n;
    double *R = (double *)malloc(sizeof(double) * (size_t)n * (size_t)(nrhs > 0 ? nrhs : 1));
    double *bwd = (double *)malloc(sizeof(double) * (size_t)(nrhs > 0 ? nrhs : 1));
    double *zprev = (double *)calloc((size_t)(nrhs > 0 ? nrhs : 1), sizeof(double));
    double anorm = or_dnorm_inf(n, n, A, lda);
    if (factor_prec == 32) {
        float *W = (float *)malloc(sizeof(float) * (nn ? nn : 1));
        float *Z = (float *)malloc(sizeof(float) * (size_t)n);
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) W[IDX(i, j, n)] = (float)A[IDX(i, j, lda)];
        if (or_spotrf(n, W, n) != 0) { flags |= OR_BREAKDOWN; fail = 1; }
        if (!fail) {
            for (int c = 0; c < nrhs; ++c) {
                double bn = 0.0;
                for (int i = 0; i < n; ++i) bn = fmax(bn, fabs(B[IDX(i, c, ldb)]));
                double s = pow2_ceil(bn);
                for (int i = 0; i < n; ++i) Z[i] = (float)(B[IDX(i, c, ldb)] / s);
                or_spotrs(n, 1, W, n, Z, n);
                for (int i = 0; i < n; ++i) X[IDX(i, c, ldx)] = (double)Z[i] * s;
            }
            double *zlast = (double *)calloc((size_t)(nrhs > 0 ? nrhs : 1), sizeof(double));
            for (int c = 0; c < nrhs; ++c) {
                double xn = 0.0;
                for (int i = 0; i < n; ++i) xn = fmax(xn, fabs(X[IDX(i, c, ldx)]));
                zlast[c] = xn;
            }
            for (;;) {
                or_dresidual(n, nrhs, A, lda, X, ldx, B, ldb, R, n);
                int done = 1, nonfinite = 0, stalled = 0;
                for (int c = 0; c < nrhs; ++c) {
                    double rn = 0.0, xn = 0.0, bn = 0.0;
                    for (int i = 0; i < n; ++i) {
                        rn = fmax(rn, fabs(R[IDX(i, c, n)]));
                        xn = fmax(xn, fabs(X[IDX(i, c, ldx)]));
                        bn = fmax(bn, fabs(B[IDX(i, c, ldb)]));
                        if (!isfinite(R[IDX(i, c, n)])) nonfinite = 1;
                    }
                    double den = anorm * xn + bn;
                    bwd[c] = den > 0.0 ? rn / den : (rn > 0.0 ? INFINITY : 0.0);
                    int stagnant = iter >= 2 && zlast[c] > stall_ratio * zprev[c];
                    int at_floor = bwd[c] == 0.0 || bwd[c] <= 2.0 * 0x1p-53 || zlast[c] <= 4.0 * 0x1p-53 * xn || stagnant;
                    if (!(bwd[c] <= tol && at_floor)) done = 0;
                    if (!(bwd[c] <= tol) && stagnant) stalled = 1;
                }
                if (nonfinite) { flags |= OR_BREAKDOWN; fail = 1; break; }
                if (done) break;
                if (stalled) { flags |= OR_STALLED; fail = 1; break; }
                if (iter >= itermax) {
                    int ok = 1;
                    for (int c = 0; c < nrhs; ++c) if (!(bwd[c] <= tol)) ok = 0;
                    if (!ok) fail = 1;
                    break;
                }
                for (int c = 0; c < nrhs; ++c) {
                    double rn = 0.0;
                    for (int i = 0; i < n; ++i) rn = fmax(rn, fabs(R[IDX(i, c, n)]));
                    double s = pow2_ceil(rn);
                    for (int i = 0; i < n; ++i) Z[i] = (float)(R[IDX(i, c, n)] / s);
                    or_spotrs(n, 1, W, n, Z, n);
                    double zn = 0.0;
                    for (int i = 0; i < n; ++i) {
                        double z = (double)Z[i] * s;
                        X[IDX(i, c, ldx)] += z;
                        zn = fmax(zn, fabs(z));
                    }
                    zprev[c] = zlast[c];
                    zlast[c] = zn;
                }
                ++iter;
            }
            free(zlast);
        }
        free(W);
        free(Z);
    }
    if (factor_prec != 32 || (fail && allow_fallback)) {
        double *F = (double *)malloc(sizeof(double) * (nn ? nn : 1));
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) F[IDX(i, j, n)] = A[IDX(i, j, lda)];
        info = or_dpotrf(n, F, n);
        if (info == 0) {
            for (int c = 0; c < nrhs; ++c)
                for (int i = 0; i < n; ++i) X[IDX(i, c, ldx)] = B[IDX(i, c, ldb)];
            or_dpotrs(n, nrhs, F, n, X, ldx);
            for (int k = 0; k < 5; ++k) {
                or_dresidual(n, nrhs, A, lda, X, ldx, B, ldb, R, n);
                or_dpotrs(n, nrhs, F, n, R, n);
                for (int c = 0; c < nrhs; ++c)
                    for (int i = 0; i < n; ++i) X[IDX(i, c, ldx)] += R[IDX(i, c, n)];
                or_bwd_err(n, nrhs, A, lda, X, ldx, B, ldb, bwd);
                int done = 1;
                for (int c = 0; c < nrhs; ++c)
                    if (!(bwd[c] <= tol)) done = 0;
                if (done) break;
            }
        }
        if (factor_prec == 32) { flags |= OR_FALLBACK; iter = -1; }
        free(F);
    }
    or_bwd_err(n, nrhs, A, lda, X, ldx, B, ldb, bwd);
    double worst = 0.0;
    for (int c = 0; c < nrhs; ++c)
        if (bwd[c] > worst || isnan(bwd[c])) worst = bwd[c];
    *iter_out = iter;
    *flags_out = flags;
    *bwd_out = worst;
    free(R);
    free(bwd);
    free(zprev);
    return info;
}

/* ------------------------------------------------------------------ */
/* Condition numbers (Section 4: refinement converges while             */
/* kappa * eps_s < 1).                                                  */
/* ------------------------------------------------------------------ */

/* kappa_inf(A) = ||A||_inf ||A^{-1}||_inf with A^{-1} formed column by
 * column from an FP64 LU (n solves).  Returns +inf if A is singular. */
/* ------------------------------------------------------------------ */
/* Iterative refinement with an extra-precise residual (Section 5,      */
/* QDGESV): FP64 LU with partial pivoting, x_0 from it, then           */
/*   r = b - A x   with x = xhi + xlo and the sum carried in            */
/*                 double-double (two-products and two-sums, columns in  */
/*                 order), rounded to FP64,                              */
/*   z = (LU)^{-1} P r in FP64,                                          */
/*   x = x + z     in double-double (two-sum, renormalised),             */
/* until the last correction is below 2^-100 ||x||inf or stopped         */
/* shrinking (||z_k|| > ||z_{k-1}|| / 2 for k >= 2), at most itermax     */
/* corrections.  Returns info of the LU (> 0: singular); *iter_out the   */
/* corrections applied (-1 when itermax was reached first).             */
/* ------------------------------------------------------------------ */
int or_gesv_dd(int n, int nrhs, const double *A, int lda, const double *B, int ldb,
               double *Xhi, double *Xlo, int ldx, int itermax, int *iter_out) {
    size_t nn = (size_t)n * (size_t)n;
    double *F = (double *)malloc(sizeof(double) * (nn ? nn : 1));
    int *ipiv = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    double *r = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) F[IDX(i, j, n)] = A[IDX(i, j, lda)];
    const int info = or_dgetrf(n, F, n, ipiv);
    int worst_iter = 0;
    if (info == 0) {
        for (int c = 0; c < nrhs; ++c) {
            double *xh = &Xhi[IDX(0, c, ldx)], *xl = &Xlo[IDX(0, c, ldx)];
            const double *b = &B[IDX(0, c, ldb)];
            for (int i = 0; i < n; ++i) { xh[i] = b[i]; xl[i] = 0.0; }
            or_dgetrs(n, 1, F, n, ipiv, xh, n);
            double zprev = 0.0, znorm = 0.0;
            for (int i = 0; i < n; ++i) znorm = fmax(znorm, fabs(xh[i]));
            int it = 0;
            for (;;) {
                double xnorm = 0.0;
                for (int i = 0; i < n; ++i) xnorm = fmax(xnorm, fabs(xh[i]));
                /* r = b - A (xh + xl): double-double sum of the products */
                double rnorm = 0.0;
#pragma omp parallel for schedule(static) if (n > 256)
                for (int i = 0; i < n; ++i) {
                    double s = 0.0, comp = 0.0;
                    for (int j = 0; j < n; ++j) {
                        double p, ep, t, es;
                        two_prod(A[IDX(i, j, lda)], xh[j], &p, &ep);
                        two_sum(s, p, &t, &es);
                        s = t;
                        comp += ep + es;
                        comp = fma(A[IDX(i, j, lda)], xl[j], comp);
                    }
                    double d, e;
                    two_sum(b[i], -s, &d, &e);
                    r[i] = d + (e - comp);
                }
                for (int i = 0; i < n; ++i) rnorm = fmax(rnorm, fabs(r[i]));
                const int done = rnorm == 0.0 || znorm <= ldexp(1.0, -100) * xnorm ||
                                 (it >= 2 && znorm > 0.5 * zprev);
                if (done) break;
                if (it >= itermax) { it = -1; break; }
                or_dgetrs(n, 1, F, n, ipiv, r, n);
                zprev = znorm;
                znorm = 0.0;
                for (int i = 0; i < n; ++i) {
                    double s, e;
                    two_sum(xh[i], r[i], &s, &e);
                    e += xl[i];
                    const double h = s + e;
                    xh[i] = h;
                    xl[i] = e - (h - s);
                    znorm = fmax(znorm, fabs(r[i]));
                }
                ++it;
            }
            if (it < 0) worst_iter = -1;                        /* a column hit itermax */
            else if (worst_iter >= 0 && it > worst_iter) worst_iter = it;
        }
    }
    if (iter_out) *iter_out = worst_iter;
    free(F);
    free(ipiv);
    free(r);
    return info;
}

double or_kappa_inf(int n, const double *A, int lda) {
    size_t nn = (size_t)n * (size_t)n;
    double *F = (double *)malloc(sizeof(double) * (nn ? nn : 1));
    double *Inv = (double *)calloc(nn ? nn : 1, sizeof(double));
    int *ipiv = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) F[IDX(i, j, n)] = A[IDX(i, j, lda)];
    int info = or_dgetrf(n, F, n, ipiv);
    double kappa = INFINITY;
    if (info == 0) {
        for (int j = 0; j < n; ++j) Inv[IDX(j, j, n)] = 1.0;
#pragma omp parallel for schedule(dynamic, 4) if (n > 128)
        for (int j = 0; j < n; ++j) or_dgetrs(n, 1, F, n, ipiv, &Inv[IDX(0, j, n)], n);
        kappa = or_dnorm_inf(n, n, A, lda) * or_dnorm_inf(n, n, Inv, n);
    }
    free(F);
    free(Inv);
    free(ipiv);
    return kappa;
}

/* Hager's 1-norm estimator in Higham's form (Higham 1988; the algorithm
 * behind DGECON, Table 7): estimates ||A^{-1}||_1 from solves with A and
 * A^T using existing FP64 LU factors, and returns kappa_1 estimate
 * = ||A||_1 * est (a lower bound of the true kappa_1).  kappa_inf(A) =
 * kappa_1(A^T), so passing A^T estimates kappa_inf. */
/* The estimate of ||A^{-1}||_1 itself, from existing FP64 LU factors F,
 * ipiv of A.  trans = 1 estimates ||A^{-T}||_1 = ||A^{-1}||_inf instead (the
 * solves with A and A^T swap roles), so kappa_inf(A) can be estimated from
 * the factors of A without factoring A^T. */
double or_dinvnorm1_est_lu(int n, const double *F, int ldf, const int *ipiv, int trans) {
    double *x = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *y = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *z = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) x[i] = 1.0 / n;
    double est = 0.0;
    for (int it = 1; it <= 5; ++it) {
        /* y = B x with B = A^{-1} (trans = 0) or A^{-T} (trans = 1) */
        for (int i = 0; i < n; ++i) y[i] = x[i];
        if (trans) or_dgetrs_trans(n, 1, F, ldf, ipiv, y, n);
        else or_dgetrs(n, 1, F, ldf, ipiv, y, n);
        double g = 0.0;
        for (int i = 0; i < n; ++i) g += fabs(y[i]);
        if (it > 1 && g <= est) break;
        est = g;
        /* z = B^T sign(y) */
        for (int i = 0; i < n; ++i) z[i] = (y[i] >= 0.0) ? 1.0 : -1.0;
        if (trans) or_dgetrs(n, 1, F, ldf, ipiv, z, n);
        else or_dgetrs_trans(n, 1, F, ldf, ipiv, z, n);
        int j = 0;
        double zmax = fabs(z[0]), ztx = 0.0;
        for (int i = 0; i < n; ++i) {
            if (fabs(z[i]) > zmax) { zmax = fabs(z[i]); j = i; }
            ztx += z[i] * x[i];
        }
        if (it > 1 && zmax <= ztx) break;
        for (int i = 0; i < n; ++i) x[i] = 0.0;
        x[j] = 1.0;
    }
    /* Higham's alternating-sign safeguard vector */
    for (int i = 0; i < n; ++i)
        y[i] = ((i % 2) ? -1.0 : 1.0) * (1.0 + (double)i / (double)(n > 1 ? n - 1 : 1));
    if (trans) or_dgetrs_trans(n, 1, F, ldf, ipiv, y, n);
    else or_dgetrs(n, 1, F, ldf, ipiv, y, n);
    double alt = 0.0;
    for (int i = 0; i < n; ++i) alt += fabs(y[i]);
    alt = 2.0 * alt / (3.0 * n);
    free(x);
    free(y);
    free(z);
    return fmax(est, alt);
}

double or_kappa_1_est(int n, const double *A, int lda) {
    size_t nn = (size_t)n * (size_t)n;
    double *F = (double *)malloc(sizeof(double) * (nn ? nn : 1));
    int *ipiv = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) F[IDX(i, j, n)] = A[IDX(i, j, lda)];
    double anorm1 = 0.0;
    for (int j = 0; j < n; ++j) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += fabs(A[IDX(i, j, lda)]);
        anorm1 = fmax(anorm1, s);
    }
    double est = INFINITY;
    if (or_dgetrf(n, F, n, ipiv) == 0) est = or_dinvnorm1_est_lu(n, F, n, ipiv, 0);
    free(F);
    free(ipiv);
    return anorm1 * est;
}

/* ------------------------------------------------------------------ */
/* Rounding to the low factor precisions (round to nearest, ties to even),
 * written from the IEEE 754 / OCP definitions: bfloat16 (8 significand
 * bits, FP32 exponent range), binary16 (11 significand bits, emin -14,
 * subnormals, overflow to inf), OCP FP8 E4M3 (4 significand bits, emin -6,
 * max 448, saturating: |x| > 448 -> 448, no inf).  Used to state what
 * "operands rounded to precision p" means.                             */
/* ------------------------------------------------------------------ */
static double round_to_grid(double x, int sig_bits, int emin, double maxv, int saturate) {
    if (x == 0.0 || !isfinite(x)) return x;
    double ax = fabs(x);
    int e;
    frexp(ax, &e);          /* ax = m 2^e, m in [0.5,1): exponent of leading bit is e-1 */
    int lead = e - 1;
    if (lead < emin) lead = emin; /* subnormal range: fixed quantum */
    double q = ldexp(1.0, lead - (sig_bits - 1));
    double r = ax / q;
    double fl = floor(r);
    double frac = r - fl;
    double k;
    if (frac > 0.5) k = fl + 1.0;
    else if (frac < 0.5) k = fl;
    else k = (fmod(fl, 2.0) == 0.0) ? fl : fl + 1.0;
    double y = k * q;
    if (y > maxv) y = saturate ? maxv : INFINITY;
    return copysign(y, x);
}

double or_round_bf16(double x) {
    double y = round_to_grid(x, 8, -126, 3.38953138925153547590470800371487866880e38, 0);
    return y;
}
double or_round_fp16(double x) {
    /* values at or above 65520 round to inf under RNE */
    if (isfinite(x) && fabs(x) >= 65520.0) return copysign(INFINITY, x);
    return round_to_grid(x, 11, -14, 65504.0, 0);
}
double or_round_e4m3(double x) {
    return round_to_grid(x, 4, -6, 448.0, 1);
}

/* ------------------------------------------------------------------ */
/* GMRES-based refinement (Section 2.2: right preconditioning A M u = b, */
/* x = M u, with M = (LU)^{-1} P from the low-precision factorization,  */
/* Eq. (2); flexible GMRES outer form of Algorithm 2 storing the         */
/* preconditioned vectors Z; convergence monitored at every inner step  */
/* from the Givens-rotated least-squares residual, Section 2.2).        */
/*                                                                      */
/* Outer loop (FP64): r = b - A x; stop if bwd <= tol; one GMRES cycle  */
/* of at most m steps on A d = r:                                        */
/*   beta = ||r||_2, v_1 = r / beta                                      */
/*   for k = 1..m: z_k = M v_k (FP32 solve with the FP32 factors);      */
/*                 w = A z_k (FP64); modified Gram-Schmidt against v_j;  */
/*                 h_{k+1,k} = ||w||_2; v_{k+1} = w / h_{k+1,k};         */
/*                 apply previous Givens rotations to column k of H,     */
/*                 form a new rotation, update g; |g_{k+1}| is the       */
/*                 residual norm of the small least-squares problem;     */
/*                 stop the cycle when |g_{k+1}| <= inner_tol * beta.    */
/*   solve the k x k triangular system for y; x += Z y (FP64).           */
/* Factor precision is single (the paper's eps_s).  One right-hand side */
/* at a time.  Returns the number of outer steps; *nmatvec counts the    */
/* applications of M (each is one pair of triangular solves).            */
/* ------------------------------------------------------------------ */
int or_gmres_ir(int n, const double *A, int lda, const double *b, double *x,
                int m, int outer_max, double tol, double inner_tol,
                int *nmatvec_out, double *bwd_out) {
    size_t nn = (size_t)n * (size_t)n;
    float *W = (float *)malloc(sizeof(float) * (nn ? nn : 1));
    int *ipiv = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    double *V = (double *)malloc(sizeof(double) * (size_t)n * (size_t)(m + 1));
    double *Z = (double *)malloc(sizeof(double) * (size_t)n * (size_t)m);
    double *H = (double *)calloc((size_t)(m + 1) * (size_t)m, sizeof(double));
    double *cs = (double *)malloc(sizeof(double) * (size_t)m);
    double *sn = (double *)malloc(sizeof(double) * (size_t)m);
    double *g = (double *)malloc(sizeof(double) * (size_t)(m + 1));
    double *yv = (double *)malloc(sizeof(double) * (size_t)m);
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    float *t = (float *)malloc(sizeof(float) * (size_t)n);
    int nmv = 0, outer = 0;
    double bwd = INFINITY;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) W[IDX(i, j, n)] = (float)A[IDX(i, j, lda)];
    int sinfo = or_sgetrf(n, W, n, ipiv);
    double anorm = or_dnorm_inf(n, n, A, lda);
    double bn = 0.0;
    for (int i = 0; i < n; ++i) bn = fmax(bn, fabs(b[i]));
    if (sinfo == 0) {
        /* x_0 = M b */
        double s = pow2_ceil(bn);
        for (int i = 0; i < n; ++i) t[i] = (float)(b[i] / s);
        or_sgetrs(n, 1, W, n, ipiv, t, n);
        for (int i = 0; i < n; ++i) x[i] = (double)t[i] * s;
        for (outer = 0; outer <= outer_max; ++outer) {
            or_dresidual(n, 1, A, lda, x, n, b, n, r, n);
            double rn = 0.0, xn = 0.0;
            for (int i = 0; i < n; ++i) { rn = fmax(rn, fabs(r[i])); xn = fmax(xn, fabs(x[i])); }
            bwd = rn / (anorm * xn + bn);
            if (bwd <= tol || outer == outer_max) break;
            double beta = 0.0;
            for (int i = 0; i < n; ++i) beta += r[i] * r[i];
            beta = sqrt(beta);
            for (int i = 0; i < n; ++i) V[i] = r[i] / beta;
            for (int i = 0; i <= m; ++i) g[i] = 0.0;
            g[0] = beta;
            int k;
            for (k = 0; k < m; ++k) {
                /* z_k = M v_k in single precision, with the v scaled to
                 * unit infinity norm magnitude by a power of two */
                double vn = 0.0;
                for (int i = 0; i < n; ++i) vn = fmax(vn, fabs(V[IDX(i, k, n)]));
                double sv = pow2_ceil(vn);
                for (int i = 0; i < n; ++i) t[i] = (float)(V[IDX(i, k, n)] / sv);
                or_sgetrs(n, 1, W, n, ipiv, t, n);
                ++nmv;
                for (int i = 0; i < n; ++i) Z[IDX(i, k, n)] = (double)t[i] * sv;
                /* w = A z_k (FP64) */
                double *w = &V[IDX(0, k + 1, n)];
                for (int i = 0; i < n; ++i) w[i] = 0.0;
                for (int j = 0; j < n; ++j) {
                    double zj = Z[IDX(j, k, n)];
                    for (int i = 0; i < n; ++i) w[i] += A[IDX(i, j, lda)] * zj;
                }
                /* modified Gram-Schmidt */
                for (int j = 0; j <= k; ++j) {
                    double h = 0.0;
                    for (int i = 0; i < n; ++i) h += w[i] * V[IDX(i, j, n)];
                    H[IDX(j, k, m + 1)] = h;
                    for (int i = 0; i < n; ++i) w[i] -= h * V[IDX(i, j, n)];
                }
                double hn = 0.0;
                for (int i = 0; i < n; ++i) hn += w[i] * w[i];
                hn = sqrt(hn);
                H[IDX(k + 1, k, m + 1)] = hn;
                if (hn > 0.0)
                    for (int i = 0; i < n; ++i) w[i] /= hn;
                /* previous rotations on column k */
                for (int j = 0; j < k; ++j) {
                    double a = H[IDX(j, k, m + 1)], c = H[IDX(j + 1, k, m + 1)];
                    H[IDX(j, k, m + 1)] = cs[j] * a + sn[j] * c;
                    H[IDX(j + 1, k, m + 1)] = -sn[j] * a + cs[j] * c;
                }
                double a = H[IDX(k, k, m + 1)], c = H[IDX(k + 1, k, m + 1)];
                double den = hypot(a, c);
                if (den == 0.0) { cs[k] = 1.0; sn[k] = 0.0; }
                else { cs[k] = a / den; sn[k] = c / den; }
                H[IDX(k, k, m + 1)] = cs[k] * a + sn[k] * c;
                H[IDX(k + 1, k, m + 1)] = 0.0;
                g[k + 1] = -sn[k] * g[k];
                g[k] = cs[k] * g[k];
                if (fabs(g[k + 1]) <= inner_tol * beta || hn == 0.0) { ++k; break; }
            }
            /* back substitution H(0:k,0:k) y = g(0:k) */
            for (int i = k - 1; i >= 0; --i) {
                double s2 = g[i];
                for (int j = i + 1; j < k; ++j) s2 -= H[IDX(i, j, m + 1)] * yv[j];
                yv[i] = s2 / H[IDX(i, i, m + 1)];
            }
            for (int j = 0; j < k; ++j)
                for (int i = 0; i < n; ++i) x[i] += Z[IDX(i, j, n)] * yv[j];
        }
    }
    *nmatvec_out = nmv;
    *bwd_out = bwd;
    free(W); free(ipiv); free(V); free(Z); free(H); free(cs); free(sn);
    free(g); free(yv); free(r); free(t);
    return sinfo != 0 ? -1 : outer;
}
