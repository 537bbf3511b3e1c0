/*
 * mpsolve.h -- C ABI of the GB300 mixed-precision iterative-refinement solver.
 *
 * Method: Baboulin, Buttari, Dongarra, Kurzak, Langou, Langou, Luszczek,
 * Tomov, "Accelerating Scientific Computations with Mixed Precision
 * Algorithms".  The problem statement is Section 2.1: given A (n x n) and
 * b in FP64, factor PA = LU in a lower precision, then refine
 * x_k = x_{k-1} + z_k with the residual r_k = b - A x_{k-1} and the update
 * computed in FP64 (Algorithm 1).  Section 3.1.1 maps the steps onto
 * LAPACK's SGETRF/SGETRS (general) and SPOTRF/SPOTRS (SPD); Section 4 gives
 * the fallback to a full FP64 solve when kappa(A) * eps_s >= 1.
 *
 * Conventions shared by every entry point:
 *   - Matrices are column-major with a leading dimension (LAPACK layout).
 *   - Pointers named d* are DEVICE pointers owned by the caller; pointers
 *     named h* are HOST pointers owned by the caller.  The library never
 *     allocates device memory: scratch space comes from the caller through
 *     (work, work_bytes), sized by the matching *_workspace_bytes query.
 *   - A and B are read-only.  X is output-only and must not overlap A or B.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is stream-ordered; a call returns after reading back the
 *     small status block (iterations, flags), so X is valid on return.  The
 *     LU factorization forks its leaf pipeline onto two internal streams of
 *     the library (one of high, one of low priority, created on a device's
 *     first factorization) and joins them back into `stream` by events, so
 *     the ordering with respect to `stream` is unchanged.
 *   - Pivots are LAPACK style: int32, 1-based, row i was exchanged with row
 *     ipiv[i], applied for i = 0..n-1 in order.
 *   - Return value: 0 success; -i if argument i (1-based) is illegal
 *     (including a workspace that is too small); +i if the FP64 fallback
 *     factorization met an exact zero pivot U(i,i) (A singular); values
 *     <= -1000 report a CUDA error (-1000 - cudaError_t); mp_last_error()
 *     gives the text.
 *   - The library runs on the current CUDA device only and needs sm_103a.
 *     Not thread-safe for concurrent calls that share a workspace.
 */
#ifndef MPSOLVE_H
#define MPSOLVE_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define MP_API __attribute__((visibility("default")))
#else
#define MP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Precision of the O(n^3) factorization (Algorithm 1 step 1 at eps_s). */
typedef enum {
    MP_PREC_FP32 = 0,   /* all factorization arithmetic in FP32 (the paper's single) */
    MP_PREC_FP16X3 = 1, /* trailing-update operands split into two fp16 parts (hi + lo, power-of-two
                           scaled), three tensor-core products hi*hi + hi*lo + lo*hi with FP32
                           accumulation: about FP32 accuracy at fp16 tensor-core speed */
    MP_PREC_BF16 = 2,   /* trailing-update operands rounded to bfloat16, FP32 accumulation */
    MP_PREC_FP16 = 3,   /* trailing-update operands rounded to binary16, FP32 accumulation */
    MP_PREC_E4M3 = 4,   /* trailing-update operands scaled by a power of two per 128 x 128 block
                           (block max below 2^8) and rounded to FP8 E4M3 (round to nearest even,
                           saturating at 448); each 128-wide K-block's product is formed on the
                           tensor cores (tcgen05 kind::f8f6f4) with FP32 accumulation and unscaled
                           by its two blocks' scales */
    MP_PREC_FP64 = 5    /* no low precision: the plain double-precision solve that the paper
                           measures its speedups against (Section 3, Table 3: DGETRF + DGETRS,
                           DPOTRF + DPOTRS), FP64 factors on the GPU, x_0 from them and the same
                           acceptance test (FP64 corrections if x_0 misses it).  mp_gesv and
                           mp_posv only; the FALLBACK flag is never set and iter counts the FP64
                           corrections.  The other entry points reject it. */
} mp_prec;

/* Refinement scheme. */
typedef enum {
    MP_REFINE_CLASSICAL = 0, /* Algorithm 1 (Section 2.1) */
    MP_REFINE_GMRES = 1,     /* FGMRES preconditioned by the low-precision LU
                                (right preconditioning, Section 2.2; Section 4) */
    MP_REFINE_AUTO = 2       /* classical, switching to GMRES when it stalls */
} mp_refine;

/* Result flags (mp_stats.flags). */
#define MP_FLAG_FALLBACK 1u       /* the answer came from the FP64 re-factorization */
#define MP_FLAG_STALLED 2u        /* classical refinement stalled */
#define MP_FLAG_LOWP_BREAKDOWN 4u /* zero/non-finite low-precision pivot or non-positive
                                     Cholesky pivot */
#define MP_FLAG_NONFINITE_INPUT 8u
#define MP_FLAG_TIMEOUT 16u       /* a bounded device-side wait gave up */
#define MP_FLAG_GMRES_USED 32u
#define MP_FLAG_NOT_CONVERGED 64u /* no convergence and fallback disabled */

typedef struct {
    int prec;            /* mp_prec, default MP_PREC_FP32 */
    int refine;          /* mp_refine, default MP_REFINE_CLASSICAL */
    int itermax;         /* maximum corrections (default 30; 30 unconverged = failure, Section 4) */
    double tol;          /* backward-error target per column (default 1e-14) */
    int gmres_restart;   /* inner steps per GMRES cycle (default 30) */
    double gmres_tol;    /* relative inner residual target (default 1e-6) */
    double stall_ratio;  /* stall if ||z_k|| > stall_ratio * ||z_{k-1}|| (default 0.5) */
    int allow_fallback;  /* re-factor in FP64 on breakdown/stall/non-convergence (default 1) */
    int nb_outer;        /* outer block width of the factorization (0 = auto; 32..1024) */
    int nb_inner;        /* reserved (0 = auto) */
} mp_opts;

typedef struct {
    int iter;            /* corrections applied (>= 0), or -1 if the FP64 fallback answered */
    unsigned flags;      /* MP_FLAG_* */
    int info;            /* low-precision factorization: first zero pivot (1-based) or 0 */
    int n_precond;       /* applications of the low-precision solve (LU)^{-1} P */
    double bwd_err;      /* max over columns of ||r||inf / (||A||inf ||x||inf + ||b||inf),
                            as seen by the last convergence test */
    int nhist;           /* entries in hist */
    double hist[32];     /* max backward error before each correction */
    float ms_convert, ms_factor, ms_refine, ms_fallback; /* phase times (0 unless timing on) */
} mp_stats;

/* Fills *opts with the defaults listed above. */
MP_API void mp_default_opts(mp_opts *opts);

/* Text of the last error raised on this thread ("" if none). */
MP_API const char *mp_last_error(void);

/* ------------------------------------------------------------------------
 * Drivers (Algorithm 1, Section 2.1; LAPACK mapping Section 3.1.1).
 * ------------------------------------------------------------------------ */

/* Bytes of device workspace mp_gesv needs for (n, nrhs, opts). */
MP_API size_t mp_gesv_workspace_bytes(int n, int nrhs, const mp_opts *opts);

/* Solve A X = B for general A: factor PA = LU at opts->prec, refine in
 * FP64 until every column's normwise backward error <= opts->tol, or fall
 * back to an FP64 LU solve.  dA: n x n FP64 (lda >= max(1,n)); dB, dX:
 * n x nrhs FP64; dipiv: n int32 (output, LAPACK 1-based; the FP64 pivots
 * when the fallback answered); work: device scratch of work_bytes >=
 * mp_gesv_workspace_bytes().  stats may be NULL.  Arguments are numbered
 * 1..14 in order for the -i error convention. */
MP_API int mp_gesv(int n, int nrhs, const double *dA, int lda, const double *dB, int ldb,
            double *dX, int ldx, int32_t *dipiv, void *work, size_t work_bytes,
            const mp_opts *opts, mp_stats *stats, void *stream);

/* Same as mp_gesv but with HOST A, B, X and ipiv: the call copies A and B to
 * the device workspace, solves, and copies X and ipiv back (the copies are
 * part of the call).  work must hold mp_gesv_host_workspace_bytes(). */
MP_API size_t mp_gesv_host_workspace_bytes(int n, int nrhs, const mp_opts *opts);
MP_API int mp_gesv_host(int n, int nrhs, const double *hA, int lda, const double *hB, int ldb,
                 double *hX, int ldx, int32_t *hipiv, void *work, size_t work_bytes,
                 const mp_opts *opts, mp_stats *stats, void *stream);

/* Symmetric positive definite A (Section 3.1.1: SPOTRF/SPOTRS for the
 * factorization and solves, DSYMM for the residual; Section 6): factor
 * A = L L^T at opts->prec from the LOWER triangle of dA (the strict upper
 * triangle is never read), refine in FP64 with the residual computed from
 * the lower triangle, or fall back to an FP64 Cholesky solve.  A
 * non-positive pivot of the low-precision factorization sets
 * MP_FLAG_LOWP_BREAKDOWN (stats->info = order of the leading minor); if the
 * FP64 factorization also meets one, the return value is that order (> 0:
 * A is not positive definite) and X is not a solution.  Arguments as in
 * mp_gesv without ipiv, numbered 1..13 for the -i error convention. */
MP_API size_t mp_posv_workspace_bytes(int n, int nrhs, const mp_opts *opts);
MP_API int mp_posv(int n, int nrhs, const double *dA, int lda, const double *dB, int ldb, double *dX,
                   int ldx, void *work, size_t work_bytes, const mp_opts *opts, mp_stats *stats,
                   void *stream);

/* Batched solve of many independent small systems A_i X_i = B_i (Algorithm 1
 * per system; Section 2.1's payoff discussion: small problems are where the
 * low-precision factorization pays least, so each system runs entirely on one
 * SM inside a single persistent launch).  n[i] in [0, MP_BATCH_MAX_N],
 * nrhs[i] in [0, 8]; n, nrhs, lda, ldb, ldx, iter, flags, info are HOST
 * arrays of `batch` entries; A, B, X, ipiv are HOST arrays of DEVICE
 * pointers (column-major FP64 A_i, B_i, X_i; int32 ipiv_i, LAPACK 1-based).
 * opts->prec in {FP32, BF16, FP16} (trailing-update operands rounded to p,
 * FP32 products and sums on the CUDA cores).  Per system: iter[i] =
 * corrections applied or -1 when the FP64 fallback answered, flags[i] =
 * MP_FLAG_*, info[i] = first zero pivot of the FP64 factorization (> 0:
 * singular) or 0; iter, flags and info may be NULL.  The call returns after
 * the results are on the host.  Returns 0 or -i for an illegal argument i
 * (1..17 in order). */
#define MP_BATCH_MAX_N 512
MP_API size_t mp_gesv_batched_workspace_bytes(int batch, const int *n, const int *nrhs, const mp_opts *opts);
MP_API int mp_gesv_batched(int batch, const int *n, const int *nrhs, const double *const *A, const int *lda,
                           const double *const *B, const int *ldb, double *const *X, const int *ldx,
                           int32_t *const *ipiv, int *iter, unsigned *flags, int *info, void *work,
                           size_t work_bytes, const mp_opts *opts, void *stream);

/* Tile schedule of the batched solver (no counterpart in the paper): the
 * panel width (8 or 16 columns) of each system's low-precision
 * factorization by range of n.  Range i covers nmax[i-1] < n <= nmax[i]
 * (nmax increasing, the last >= MP_BATCH_MAX_N).  The library starts from
 * a table chosen on GB300 by the project's autotuner, which times every
 * width on each range of n and writes the table into the library's sources;
 * mp_batched_set_schedule replaces it for the process (count = 0 restores
 * the built-in table) and is what the autotuner uses to time candidates.
 * The schedule is process-wide: change it only while no batched solve is in
 * flight.  Returns 0 or -i for an illegal argument i.  mp_batched_get_schedule
 * copies up to cap entries and sets *count to the number of ranges. */
MP_API int mp_batched_set_schedule(int count, const int *nmax, const int *nb);
MP_API int mp_batched_get_schedule(int cap, int *count, int *nmax, int *nb);

/* Solve A X = B to more than FP64 accuracy by refinement with an
 * extra-precise residual (Section 5, QDGESV: an FP64 LU factorization, then
 * iterative refinement whose residual b - A x is computed, and whose solution
 * is kept, in a precision beyond FP64; Tables 6 and 7).  Here the extended
 * precision is double-double: X is returned as the unevaluated sum
 * Xhi + Xlo of two FP64 arrays (|Xlo| <= ulp(Xhi)/2).  A (n x n) and B
 * (n x nrhs) are FP64 column-major DEVICE arrays read as exact values; the
 * factorization is FP64 LU with partial pivoting (dipiv: n int32, LAPACK
 * 1-based, output); x_0 is the FP64 solve and each step computes
 * r = b - A (xhi + xlo) accumulated in double-double (error-free
 * two-products and two-sums, rounded to FP64 at the end), solves for z with
 * the FP64 factors and adds it in double-double.  A column stops when its
 * last correction is below 2^-100 ||x||inf or stopped shrinking (||z_k|| >
 * ||z_{k-1}|| / 2 for k >= 2: the limiting accuracy), the loop at itermax
 * corrections (MP_FLAG_NOT_CONVERGED).  stats (optional): iter = corrections,
 * hist/bwd_err = the FP64 normwise backward error of each residual,
 * ms_convert / ms_factor / ms_refine = phase times.  Returns 0, -i for an
 * illegal argument i (1..15), +i for an exact zero pivot U(i,i) (A singular;
 * X is not computed), or a CUDA error (<= -1000).  work: DEVICE scratch of
 * mp_gesv_dd_workspace_bytes(n, nrhs) bytes. */
MP_API size_t mp_gesv_dd_workspace_bytes(int n, int nrhs);
MP_API int mp_gesv_dd(int n, int nrhs, const double *dA, int lda, const double *dB, int ldb, double *dXhi,
                      double *dXlo, int ldx, int32_t *dipiv, int itermax, void *work, size_t work_bytes,
                      mp_stats *stats, void *stream);

/* Linear least squares min ||b - A x||_2 for A m x n (m >= n, full column
 * rank) by mixed-precision refinement of the augmented system (Section 6
 * names least squares among the algorithms the approach extends to; the
 * augmented formulation is Bjorck's):
 *     [ alpha I   A ] [ r / alpha ]   [ b ]
 *     [ A^T       0 ] [ x         ] = [ 0 ]
 * The (m + n)-order system is built in the workspace and solved by mp_gesv
 * with opts (low-precision LU with partial pivoting, FP64 residual and
 * refinement, FP64 fallback), which gives x and the residual r = b - A x in
 * FP64.  alpha: a power of two (exact scaling), 0 = automatic (the power of
 * two nearest ||A||_F / sqrt(8 n), about sigma_min / sqrt(2) for a
 * well-conditioned A, where the augmented matrix's condition number is about
 * 2 kappa_2(A)).  dA: m x n, dB: m x nrhs, dX: n x nrhs, dR (optional, NULL
 * to skip): m x nrhs, all FP64 column-major DEVICE arrays.  stats: those of
 * the augmented solve.  Returns 0, -i for an illegal argument i (1..17), +i
 * when the FP64 factorization of the augmented matrix met a zero pivot
 * (A rank deficient), or a CUDA error (<= -1000).  m + n <= 65536. */
MP_API size_t mp_gels_workspace_bytes(int m, int n, int nrhs, const mp_opts *opts);
MP_API int mp_gels(int m, int n, int nrhs, const double *dA, int lda, const double *dB, int ldb, double *dX,
                   int ldx, double *dR, int ldr, double alpha, void *work, size_t work_bytes, const mp_opts *opts,
                   mp_stats *stats, void *stream);

/* Adjoint of the solve (reverse-mode derivative of X = A^{-1} B; the paper
 * has no counterpart).  Given the FP64 cotangent G = dL/dX (n x nrhs),
 * computes Bbar = A^{-T} G (n x nrhs) and Abar = -Bbar X^T (n x n, FP64,
 * column-major ldab) from the factors that the preceding mp_gesv or mp_posv
 * call left in `work`: the transposed low-precision solves use W^T (built in
 * adj_work), and the transposed system is refined in FP64 against A^T by the
 * Algorithm 1 loop with the same tol/itermax/stall rules (for mp_posv,
 * A^T = A and the forward factors are used as they are).  work and opts
 * (prec, nb_outer, allow_fallback) must be those of the forward call, which
 * must have returned 0, and no other solve may have used `work` since; dX
 * is the forward solution.  adj_work: mp_gesv_adjoint_workspace_bytes()
 * (unused after mp_posv, may be NULL then).  stats->flags gets
 * MP_FLAG_FALLBACK when the forward call's FP64 factors were used and
 * MP_FLAG_NOT_CONVERGED when the refinement stopped short of tol.
 * Arguments are numbered 1..19 in order for the -i error convention. */
MP_API size_t mp_gesv_adjoint_workspace_bytes(int n, const mp_opts *opts);
MP_API int mp_gesv_adjoint(int n, int nrhs, const double *dA, int lda, const double *dX, int ldx,
                           const double *dG, int ldg, double *dBbar, int ldbb, double *dAbar, int ldab,
                           void *work, size_t work_bytes, void *adj_work, size_t adj_bytes,
                           const mp_opts *opts, mp_stats *stats, void *stream);

/* Allocation-free variant of mp_gesv (the paper has no counterpart; this is
 * a deployment convenience).  Some callers may not call cudaMalloc: services
 * that fix their device memory at start-up and forbid allocation afterwards
 * (an allocation can synchronize the device and can fail under memory
 * pressure), and plug-ins whose host framework owns every device allocation
 * and hands them no allocator.  This entry point takes
 * its scratch from a static device array of MP_NOALLOC_SCRATCH_BYTES that is
 * part of the library image: every GPU that loads the library holds that
 * memory until the process exits.  The caller still passes A, B, X and ipiv
 * (device pointers, as for mp_gesv); the call allocates nothing.
 *   - Sizes whose mp_gesv_workspace_bytes(n, nrhs, opts) exceed the array
 *     return -1 with an explanatory mp_last_error().
 *   - The first call on a device looks up the array's device address and
 *     creates the internal streams (with that device current); make that
 *     first call before any stream capture.  The address is kept for the
 *     life of the process: do not call this entry point again on a device
 *     after cudaDeviceReset (or any other teardown of its primary context).
 *   - Every call on a device shares the one array and it keeps the previous
 *     call's contents; the solver re-initializes everything it needs.  Calls
 *     that overlap on the GPU (different streams or host threads) race on the
 *     array: serialize them.
 *   - Phase times in mp_stats are not measured (left 0). */
#define MP_NOALLOC_SCRATCH_BYTES (64u * 1024u * 1024u)
MP_API size_t mp_noalloc_scratch_bytes(void);
MP_API int mp_gesv_noalloc(int n, int nrhs, const double *dA, int lda, const double *dB, int ldb,
                           double *dX, int ldx, int32_t *dipiv, const mp_opts *opts,
                           mp_stats *stats, void *stream);

/* ------------------------------------------------------------------------
 * Sparse systems: the mixed-precision inner-outer iterative method of
 * Section 2.2 (Algorithm 2), FGMRES(m_out)-GMRES_SP(m_in).
 * The matrix is CSR on the DEVICE, owned by the caller: indptr (n + 1 int32,
 * indptr[0] = 0, non-decreasing, indptr[n] = nnz), indices (nnz int32 column
 * numbers in [0, n)) and values (nnz FP64).  The library does not check the
 * structure (it is device data); a malformed one reads out of bounds.
 * ------------------------------------------------------------------------ */

/* Inner solver of the preconditioner. */
typedef enum {
    MP_INNER_FP32 = 0, /* GMRES_SP: one cycle of GMRES(m_in) on the FP32-rounded values, every
                          operation of the cycle in FP32 (the paper's mixed-precision method) */
    MP_INNER_FP64 = 1, /* GMRES_DP: the same cycle in FP64 (the paper's FGMRES-GMRES_DP, Fig. 5 left) */
    MP_INNER_NONE = 2  /* no preconditioner: plain restarted GMRES(m_out) in FP64 (Fig. 5 right) */
} mp_inner;

typedef struct {
    int m_out;       /* outer restart: FGMRES steps per cycle, 1..320 (default 20) */
    int m_in;        /* inner restart: GMRES steps of one preconditioner cycle, 1..320 (default 30) */
    int inner;       /* mp_inner (default MP_INNER_FP32) */
    int max_cycles;  /* restarts of the outer method (default 100) */
    double tol;      /* target normwise backward error ||b - Ax||inf / (||A||inf ||x||inf + ||b||inf)
                        (default 1e-14) */
} mp_sparse_opts;

typedef struct {
    int cycles;       /* outer restart cycles run */
    int outer_steps;  /* FGMRES steps over all cycles */
    int inner_steps;  /* GMRES steps of all preconditioner cycles */
    unsigned flags;   /* MP_FLAG_NOT_CONVERGED (tol not reached in max_cycles), MP_FLAG_TIMEOUT */
    double bwd_err;   /* backward error of the returned x */
    int nhist;        /* entries in hist */
    double hist[32];  /* backward error at the start of each cycle */
} mp_sparse_stats;

/* Fills *opts with the defaults listed above. */
MP_API void mp_sparse_default_opts(mp_sparse_opts *opts);

/* Solve A x = b (A n x n sparse, CSR as above; b, x: n FP64 DEVICE vectors)
 * by Algorithm 2 (Section 2.2) from x_0 = 0: each outer cycle computes
 * r = b - A x in FP64 and stops when the backward error is <= tol; otherwise
 * it runs up to m_out flexible-GMRES steps in FP64 whose preconditioner z_k is
 * one cycle of the inner GMRES for A z = v_k (from z = 0), orthogonalises
 * A z_k in FP64, ends early once the least-squares residual estimate shows
 * the accuracy test will pass, and updates x = x + Z y.  Each cycle is one
 * cooperative launch with bounded grid barriers (a timeout sets
 * MP_FLAG_TIMEOUT and ends the solve); the call returns after the last cycle.
 * work: DEVICE scratch of mp_fgmres_workspace_bytes(n, nnz, opts) bytes.
 * stats may be NULL.  Returns 0, -i for an illegal argument i (1..12 in
 * order), or a CUDA error (<= -1000). */
MP_API size_t mp_fgmres_workspace_bytes(int n, long long nnz, const mp_sparse_opts *opts);
MP_API int mp_fgmres(int n, long long nnz, const int32_t *d_indptr, const int32_t *d_indices,
                     const double *d_values, const double *d_b, double *d_x, void *work, size_t work_bytes,
                     const mp_sparse_opts *opts, mp_sparse_stats *stats, void *stream);

/* Steps of Algorithm 2, for testing.  mp_sparse_gmres_cycle: one cycle of
 * GMRES(m) for A z = v from z = 0 in precision inner (MP_INNER_FP32: values and
 * v rounded to FP32, every operation in FP32; MP_INNER_FP64), ending early at
 * breakdown or when its residual estimate is at 4 u of the working precision
 * times ||v||; z returned in FP64, *steps (host, may be NULL) = steps taken.
 * work: mp_fgmres_workspace_bytes(n, nnz, opts with m_in = m, m_out = 1).
 * mp_csr_spmv: y = A x, prec MP_PREC_FP64, or MP_PREC_FP32 (values and x
 * rounded to FP32, products and sums in FP32, y widened to FP64); x, y: n
 * FP64 DEVICE vectors.  Both return 0, -i for an illegal argument i, or a CUDA
 * error (<= -1000). */
MP_API int mp_sparse_gmres_cycle(int n, long long nnz, const int32_t *d_indptr, const int32_t *d_indices,
                                 const double *d_values, const double *d_v, double *d_z, int m, int inner,
                                 void *work, size_t work_bytes, int *steps, void *stream);
MP_API int mp_csr_spmv(int n, long long nnz, const int32_t *d_indptr, const int32_t *d_indices,
                       const double *d_values, const double *d_x, double *d_y, int prec, void *stream);

/* ------------------------------------------------------------------------
 * Steps of the hot path, exposed for testing and for callers that keep
 * the factors (Section 3.1.1: SGETRF, SGETRS, DGEMM residual, DAXPY).
 * The low-precision factors live in the caller's workspace as W, an FP32
 * ROW-major n x ldw array (ldw = mp_factor_ld(n)).
 * ------------------------------------------------------------------------ */

/* Leading dimension (in elements) of the row-major FP32 factor array W. */
MP_API int mp_factor_ld(int n);

/* Bytes of workspace needed by mp_getrf_lowp beyond W itself. */
MP_API size_t mp_getrf_workspace_bytes(int n, const mp_opts *opts);

/* W = fl32(A) stored row-major (W[i*ldw + j] = fl32(A[i + j*lda])), and
 * *d_anorm (device double) = ||A||_inf.  Sets MP_FLAG_NONFINITE_INPUT in
 * *d_flags (device uint32, OR-ed) if A has a NaN/Inf. */
MP_API int mp_convert(int n, const double *dA, int lda, float *dW, int ldw,
               double *d_anorm, uint32_t *d_flags, void *work, size_t work_bytes,
               void *stream);

/* In-place LU with partial pivoting of the row-major FP32 W (n x n, ldw),
 * trailing updates at opts->prec.  dipiv: n int32 LAPACK 1-based.
 * On return *info (host) = first zero pivot (1-based) or 0, and *flags
 * (host) has MP_FLAG_LOWP_BREAKDOWN if a pivot was zero or non-finite. */
MP_API int mp_getrf_lowp(int n, float *dW, int ldw, int32_t *dipiv, const mp_opts *opts,
                  void *work, size_t work_bytes, int *info, uint32_t *flags, void *stream);

/* In-place Cholesky A = L L^T of the row-major FP32 W (n x n, ldw a multiple
 * of 32 >= n; only the lower triangle is read), L left in the lower
 * triangle; the strict upper triangle is used as scratch (its values on
 * return are unspecified).  Trailing updates A22 -= fl_p(L21) fl_p(L21)^T at
 * opts->prec (Section 3.1.1, SPOTRF).  On return *info (host) = order of the
 * first leading minor found not positive (1-based) or 0, and *flags has
 * MP_FLAG_LOWP_BREAKDOWN in that case.  work: mp_getrf_workspace_bytes(). */
MP_API int mp_potrf_lowp(int n, float *dW, int ldw, const mp_opts *opts, void *work, size_t work_bytes,
                         int *info, uint32_t *flags, void *stream);

/* Solve with the FP32 factors (Algorithm 1 steps 5-6):
 * dZ = s * U^{-1} L^{-1} P (dR / s) computed in FP32, s = 2^ceil(log2 ||r||inf)
 * per column (exact scaling), returned in FP64.  dW must be 16-byte aligned
 * with ldw a multiple of 4 (mp_factor_ld(n) is).  dR, dZ: n x nrhs FP64
 * column-major (nrhs <= 8).  work must hold mp_getrs_workspace_bytes(n, nrhs). */
MP_API size_t mp_getrs_workspace_bytes(int n, int nrhs);
MP_API int mp_getrs_lowp(int n, int nrhs, const float *dW, int ldw, const int32_t *dipiv,
                  const double *dR, int ldr, double *dZ, int ldz, void *work,
                  size_t work_bytes, void *stream);

/* Trailing update of the blocked factorization (the O(n^3) step of
 * Algorithm 1 step 1, Section 2.1): C[M x N] -= fl_p(L)[M x K] * fl_p(U)[K x N]
 * with all three arrays FP32 ROW-major on the device (ldl >= K, ldu >= N,
 * ldc >= N; ldl, ldu, ldc multiples of 4).  prec: MP_PREC_FP32 (plain FP32
 * FMA on CUDA cores), MP_PREC_BF16 / MP_PREC_FP16 (operands rounded to
 * nearest even, FP32 accumulation on tcgen05 tensor cores), MP_PREC_FP16X3
 * (split operands, three tensor-core products), MP_PREC_E4M3 (every 128 x 128
 * block of each operand scaled by its own power of two, block max below 2^8,
 * rounded to E4M3; each K-block's product unscaled by its two blocks' scales
 * in the FP32 epilogue).  work must hold
 * mp_lowp_gemm_workspace_bytes(M, N, K, prec). */
MP_API size_t mp_lowp_gemm_workspace_bytes(int M, int N, int K, int prec);
MP_API int mp_lowp_gemm_update(int prec, int M, int N, int K, const float *dL, int ldl,
                               const float *dU, int ldu, float *dC, int ldc, void *work,
                               size_t work_bytes, void *stream);

/* dR = dB - dA dX in FP64 (Algorithm 1 step 4), all n x nrhs column-major.
 * work must hold mp_residual_workspace_bytes(n, nrhs). */
MP_API size_t mp_residual_workspace_bytes(int n, int nrhs);
MP_API int mp_residual(int n, int nrhs, const double *dA, int lda, const double *dX, int ldx,
                const double *dB, int ldb, double *dR, int ldr, void *work,
                size_t work_bytes, void *stream);

/* Self-test of failure detection (no counterpart in the paper).  Every
 * device-side wait of the library is bounded: after about one second it gives
 * up, sets MP_FLAG_TIMEOUT and the kernel returns, so the host sees an error
 * status instead of a hung GPU.  This call runs one of those waits on a
 * condition that nothing satisfies, with the caller's limit, and reports what
 * the kernel recorded.  site: 2 = the grid barrier of the triangular solves
 * (a generation that needs one arrival more than the grid has), 3 = the
 * panel kernel's mbarrier wait, 4 = the tensor-core kernels' mbarrier wait
 * (both expecting 16 bytes that nothing sends).  limit_ns in [1, 1e9].  work:
 * DEVICE scratch of mp_selftest_workspace_bytes() bytes.  On return *flags
 * (host) holds the recorded MP_FLAG_* bits, *site_out the recorded site and
 * *passed (site 2) the CTAs that got past the barrier (0 when the timeout
 * path works); any of them may be NULL.  Returns 0 once the kernel has
 * returned, -i for an illegal argument i, or a CUDA error (<= -1000). */
MP_API size_t mp_selftest_workspace_bytes(void);
MP_API int mp_selftest_wait_timeout(int site, unsigned long long limit_ns, void *work, size_t work_bytes,
                                    unsigned *flags, int *site_out, int *passed, void *stream);

/* ------------------------------------------------------------------------
 * Instrumentation (no counterpart in the paper; used by the benchmark).
 * ------------------------------------------------------------------------ */

/* Kernel classes timed by the profiler. */
#define MP_KC_PANEL 0      /* pivoted panel (cluster kernel) */
#define MP_KC_ROWMOVES 1   /* composed row exchanges */
#define MP_KC_TRSM 2       /* U12 = L11^{-1} A12 (small solves + FP32 GEMMs) */
#define MP_KC_UPDATE 3     /* trailing update A22 -= L21 U12 (outer level) */
#define MP_KC_PANELGEMM 4  /* FP32 updates inside the recursive panel */
#define MP_KC_TRSV 5       /* triangular solves with the factors */
#define MP_KC_RESIDUAL 6   /* FP64 residual */
#define MP_KC_COUNT 7

/* Enables (mask != 0) or disables event timing of the kernel classes in
 * mask (bit i = class i) on the stream each kernel is launched on, and
 * clears the accumulated records. */
MP_API void mp_profile_enable(unsigned mask);
/* Times one launch in every `every` (>= 1; default 1 = all) of each enabled
 * class, counting from the last mp_profile_enable or mp_profile_sample call,
 * so that the events add little to a latency-bound chain of launches. */
MP_API void mp_profile_sample(int every);
/* Waits for the recorded events and returns, per class, the summed kernel
 * time (ms), the number of timed launches and the summed algorithmic work of
 * those launches (flops for PANEL/TRSM/UPDATE/PANELGEMM, bytes for the
 * others).  Arrays have MP_KC_COUNT entries.  Returns 0 or a CUDA error code. */
MP_API int mp_profile_collect(double *ms, long long *launches, double *work);
/* Number of kernels this library has launched in this process so far. */
MP_API long long mp_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* MPSOLVE_H */
