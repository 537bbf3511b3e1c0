// kernels.cuh -- launchers of the device kernels (host-callable, stream-ordered).
// Every matrix argument here is ROW-major with the given leading dimension
// unless it is named col-major.
#pragma once

#include "common.cuh"

// ---- pivoted panel (panel.cu) ----------------------------------------------
template <typename T> int panel_base_width(int m);
// CTAs in the cluster of the panel kernel for a panel of height m.
template <typename T> int panel_cluster_size(int m);
// LU with partial pivoting of the m x ncols panel starting at P (row-major, ld),
// ncols <= panel_base_width<T>(m).  ipiv[j] (j < ncols) receives the global
// 1-based pivot row row0 + p + 1; moves[0 .. *nmoves) receives the composed
// row permutation of the panel as (destination row, source row) pairs
// (global row indices, at most 2 * ncols).  linv (optional): receives the
// inverse of the unit-lower ncols x ncols L11, row-major with stride
// panel_base_width<T>(m).
//
// prev (optional, prev.kb > 0): the previous leaf of the same outer panel,
// whose row moves and update the panel's columns have NOT received yet; the
// kernel applies them while loading (rows taken through the moves, then
// A -= L21 U with U = X A12, the same FMA order as launch_leaf_update) and
// writes U to the previous leaf's rows (prev.kb rows above P).
template <typename T>
struct PanelPrev {
    const T *X = nullptr;          // the previous leaf's L11^{-1}, row-major, stride xs
    const int2 *pairs = nullptr;   // its row moves (destination, source), global rows
    const int *npairs = nullptr;   // their count (device)
    int xs = 0;
    int kb = 0;                    // its width; its columns end where the panel starts
};
template <typename T>
cudaError_t launch_panel(T *P, long ld, int m, int ncols, int row0, int32_t *ipiv, int2 *moves,
                         int *nmoves, MpDevStatus *st, T *linv, PanelPrev<T> prev, cudaStream_t s);

// ---- row exchanges (blas3.cu) ---------------------------------------------
// Composes the swaps ipiv[k1..k2) (1-based rows) into a list of (dst, src)
// row moves; npairs_out receives the count (device int).  map_scratch holds
// n ints (identity on entry, restored on exit) for tall matrices.
cudaError_t launch_compose_swaps(const int32_t *ipiv, int k1, int k2, int n, int2 *pairs,
                                 int *npairs, int *map_scratch, cudaStream_t s);
// Applies the moves to columns [c0,c1) and [c2,c3) of W, and (if perm is not
// null) to the row permutation vector perm.
template <typename T>
cudaError_t launch_apply_moves(T *W, long ld, const int2 *pairs, const int *npairs, int max_pairs,
                               int c0, int c1, int c2, int c3, int *perm, cudaStream_t s);
// After a factored leaf (columns [k, k+kb), rows exchanged): U = X A12 with
// X = L11^{-1} (from the panel kernel, row-major with stride xs) on rows
// k..k+kb of the N columns starting coff after the leaf (coff a multiple of
// 4), and A22 -= L21 U on the M rows below, in one launch (kb <= 24 FP32 /
// 8 FP64, N <= 1024).  tickets: one device word per 128 columns, zero before
// the first launch (left zero).
template <typename T>
cudaError_t launch_leaf_update(T *W, long ld, int k, int kb, int coff, int N, int M, const T *X, int xs,
                               unsigned *tickets, cudaStream_t s);
// The same leaf step BEFORE the leaf's row exchange, as a persistent launch
// of `clusters` clusters of `cluster` CTAs (one CTA per SM): it applies the
// leaf's row moves (pairs, *npairs) to the updated columns, to the columns
// [0, mc1) and [mc2, mc3) and to the row permutation perm (optional).  It
// also forms, left-looking, the U rows of the previous leaf (rows
// [kp, kp+kbp)) over the trailing columns [tc0, tc1):
// U_p = Xp (A12_p - L_p U_<p) with L_p = those rows of the outer panel's
// columns [k0, kp) and U_<p = rows [k0, kp) of the trailing columns.  With
// clusters = leaf_update_rest_clusters(cluster) one cluster slot stays free
// for a concurrent panel kernel of that cluster size.  N may be 0 (moves
// only), kb may be 0 (nothing but the previous leaf's U rows), npairs may be
// null (no moves); M at most 655360.
template <typename T>
struct LeafRestArgs {
    T *W = nullptr;
    long ld = 0;
    int k = 0, kb = 0, coff = 0, N = 0, M = 0;
    const T *X = nullptr;
    int xs = 0;
    unsigned *tickets = nullptr;
    const int2 *pairs = nullptr;
    const int *npairs = nullptr;
    int mc1 = 0, mc2 = 0, mc3 = 0;
    int *perm = nullptr;
    // the previous leaf's U rows over the trailing columns (kbp = 0: none)
    const T *Xp = nullptr;
    int xps = 0, kp = 0, kbp = 0, k0 = 0, tc0 = 0, tc1 = 0;
    // optional: running max |U| of those rows (uint bits of a non-negative
    // float, NaN counted as infinite), atomically raised
    unsigned *umax = nullptr;
};
template <typename T>
cudaError_t launch_leaf_rest(const LeafRestArgs<T> &p, int clusters, int cluster, cudaStream_t s);
template <typename T> int leaf_update_rest_clusters(int cluster);
// Applies the moves to an int vector (the running row permutation).
cudaError_t launch_apply_moves_vec(int *v, const int2 *pairs, const int *npairs, int max_pairs,
                                   cudaStream_t s);

// ---- level-3 helpers (blas3.cu) ---------------------------------------------
// C[MxN] -= A[MxK] * B[KxN], SIMT FMA in T.
template <typename T>
cudaError_t launch_gemm_sub(int M, int N, int K, const T *A, long lda, const T *B, long ldb,
                            T *C, long ldc, cudaStream_t s);
// Batched C_z = beta*C_z + alpha*A_z*B_z (beta = 0 or 1), z = 0..batch-1,
// with X_z = X + (z / inner) * x_outer + (z % inner) * x_inner.
template <typename T>
cudaError_t launch_gemm_batched(int M, int N, int K, T alpha, T beta, const T *A, long lda, const T *B, long ldb,
                                T *C, long ldc, int batch, int inner, long a_outer, long a_inner, long b_outer,
                                long b_inner, long c_outer, long c_inner, cudaStream_t s);
// C[MxN] -= A[MxK] * B[NxK]^T; lower != 0 skips C tiles strictly above the
// diagonal (C square, symmetric update).
template <typename T>
cudaError_t launch_gemm_nt_sub(int M, int N, int K, const T *A, long lda, const T *B, long ldb, T *C, long ldc,
                               int lower, cudaStream_t s);
// B[m x N] <- L^{-1} B with L unit lower (m x m, ldl), m <= 64.
template <typename T>
cudaError_t launch_trsm_llnu_small(int m, int N, const T *L, long ldl, T *B, long ldb,
                                   cudaStream_t s);

// ---- conversions and norms (convert.cu) -------------------------------------
// W (row-major, ldw) = (Tout) A (col-major, lda); rowsum[i] += sum_j |a_ij|;
// non-finite -> flag.  rowsum must be zeroed first.
template <typename Tout>
cudaError_t launch_convert_transpose(int n, const double *A, long lda, Tout *W, long ldw,
                                     double *rowsum, MpDevStatus *st, cudaStream_t s);
cudaError_t launch_max_reduce(int n, const double *v, double *out, cudaStream_t s);
// Symmetric A by its lower triangle: W[r][c] = fl(a_rc) for r >= c; rowsum
// of the full symmetric |A| (accumulated, zero first).
template <typename Tout>
cudaError_t launch_convert_lower(int n, const double *A, long lda, Tout *W, long ldw, double *rowsum,
                                 MpDevStatus *st, cudaStream_t s);

// ---- Cholesky (chol.cu) --------------------------------------------------------
int potrf_leaf_width();
// Factor columns [k0, k0 + nc) of rows [k0, n) (nc <= potrf_leaf_width()),
// all earlier updates applied: diagonal block L11 L11^T and L21 = A21 L11^{-T}.
template <typename T>
cudaError_t launch_potrf_leaf(int n, int k0, int nc, T *W, long ldw, MpDevStatus *st, cudaStream_t s);
// Upper triangle of W <- transpose of its strict lower triangle.
template <typename T>
cudaError_t launch_mirror_lower(int n, T *W, long ldw, cudaStream_t s);
// Wt = W^T (n x n, row-major both).
template <typename T>
cudaError_t launch_transpose(int n, const T *W, long ldw, T *Wt, long ldwt, cudaStream_t s);

// ---- triangular solves with the factors (trsv.cu) ---------------------------
// Diagonal blocks of L and U are inverted at block size BI (1024 rows FP32,
// 512 FP64, smaller for small n); the solves then take n/BI steps.
template <typename T> int trsv_inverse_block(int n);
template <typename T> size_t trsv_inverse_bytes(int n);  // per triangle
template <typename T> size_t trsv_tmp_bytes(int n);
template <typename T> size_t trsv_sync_bytes(int n);  // counters of one solve (zeroed by the launch)
template <typename T>
cudaError_t launch_build_inverses(int n, const T *W, long ldw, T *Linv, T *Uinv, T *tmp, cudaStream_t s,
                                  bool lower_unit = true, bool upper_unit = false);
// Lower solve: Y[:,c] = L^{-1} (P r_c) / s_c with r FP64 col-major (ldr), perm
// (nullptr: identity)
// the row permutation, s_c = 2^ceil(log2 rnorm[c]).  acc: n*nrhs scratch of T;
// bar: two unsigned words, zero before first use (a grid barrier).
template <typename T>
cudaError_t launch_trsv_lower(int n, int nrhs, const T *W, long ldw, const T *Linv, const double *R, long ldr,
                              const int *perm, const double *rnorm, T *Y, long ldy, T *acc, unsigned *bar,
                              MpDevStatus *st, cudaStream_t s);
// Upper solve: Z = U^{-1} Y.
template <typename T>
cudaError_t launch_trsv_upper(int n, int nrhs, const T *W, long ldw, const T *Uinv, const T *Y, long ldy, T *Z,
                              long ldz, T *acc, unsigned *bar, MpDevStatus *st, cudaStream_t s);

// ---- FP64 residual and update (refine.cu) -----------------------------------
int residual_ksplit(int n, int nrhs);
// part[ks][c][i] partial sums of (A X)[i,c] over column chunk ks.
cudaError_t launch_residual_partial(int n, int nrhs, const double *A, long lda, const double *X,
                                    long ldx, double *part, int ksplit, cudaStream_t s);
// Symmetric A (lower triangle read): part[K][c][i] = (block column K of A) x_c
// for K < residual_sym_blocks(n); finalize with ksplit = residual_sym_blocks(n).
int residual_sym_blocks(int n);
cudaError_t launch_residual_sym_partial(int n, int nrhs, const double *A, long lda, const double *X, long ldx,
                                        double *part, cudaStream_t s);
// R = B - sum_ks part (R = A X when B is null); rnorm[c] = ||R_c||inf,
// xnorm[c] = ||X_c||inf (zeroed first).
cudaError_t launch_residual_finalize(int n, int nrhs, const double *part, int ksplit,
                                     const double *B, long ldb, const double *X, long ldx,
                                     double *R, long ldr, double *rnorm, double *xnorm,
                                     MpDevStatus *st, cudaStream_t s);
// X[:,c] (+)= s_c * Z[:,c] with s_c = 2^ceil(log2 rnorm[c]); znorm[c] = ||s_c Z_c||inf.
// scatter (optional): row i of Z goes to row scatter[i] of X (x = P^T z).
template <typename T>
cudaError_t launch_update(int n, int nrhs, const T *Z, long ldz, const double *rnorm, double *X,
                          long ldx, double *znorm, int assign, cudaStream_t s, const int *scatter = nullptr);
// R = G - A^T L (FP64, A column-major n x n: one warp per column of A, fixed
// summation order); rnorm[c] = ||R_c||inf, xnorm[c] = ||L_c||inf (zeroed first).
cudaError_t launch_residual_trans(int n, int nrhs, const double *A, long lda, const double *L, long ldl,
                                  const double *G, long ldg, double *R, long ldr, double *rnorm, double *xnorm,
                                  MpDevStatus *st, cudaStream_t s);
// Abar = -L X^T (n x n FP64 column-major), the rank-nrhs outer product of the adjoint.
cudaError_t launch_outer_neg(int n, int nrhs, const double *L, long ldl, const double *X, long ldx, double *Abar,
                             long ldab, cudaStream_t s);
// bnorm[c] = ||B_c||_inf (zeroed first)
cudaError_t launch_col_absmax(int n, int nrhs, const double *B, long ldb, double *out,
                              MpDevStatus *st, cudaStream_t s);

// ---- GMRES-based refinement pieces (refine.cu) -------------------------------
// out[j] = V[:, j] . w for j < k (FP64, column-major V)
cudaError_t launch_dots(int n, int k, const double *V, long ldv, const double *w, double *out, cudaStream_t s);
// w -= V[:, 0:k] h
cudaError_t launch_project(int n, int k, const double *V, long ldv, const double *h, double *w, cudaStream_t s);
// x += Z[:, 0:k] y; *znorm = max |Z y| (zeroed first)
cudaError_t launch_correct(int n, int k, const double *Z, long ldz, const double *y, double *x, double *znorm,
                           cudaStream_t s);
// dst = src / d
cudaError_t launch_scale(int n, const double *src, double d, double *dst, cudaStream_t s);

// ---- timeout paths of the bounded waits (self-test) --------------------------
// Each runs one of the library's bounded waits on a condition nothing
// satisfies, with the given limit, recording MP_FLAG_TIMEOUT and the site in st.
// bar: two zeroed words; passed: CTAs that got past the grid barrier;
// abort_flag: a zeroed word.
cudaError_t launch_selftest_grid_barrier(unsigned *bar, MpDevStatus *st, unsigned long long limit_ns, int *passed,
                                         cudaStream_t s);
cudaError_t launch_selftest_panel_mbar(MpDevStatus *st, unsigned long long limit_ns, cudaStream_t s);
cudaError_t launch_selftest_tc_mbar(MpDevStatus *st, const int *abort_flag, unsigned long long limit_ns,
                                    cudaStream_t s);

// ---- extra-precise refinement (dd.cu) ------------------------------------------
// Column chunks of the double-double residual (part arrays: ksplit x nrhs x n each).
int residual_dd_ksplit(int n);
// R = fl64(B - A (Xhi + Xlo)) with the residual accumulated in double-double;
// rnorm/xnorm (zeroed by the caller) = max |R|, max |Xhi| per column.
cudaError_t launch_residual_dd(int n, int nrhs, const double *A, long lda, const double *Xhi, const double *Xlo,
                               long ldx, const double *B, long ldb, double *part_hi, double *part_lo, int ksplit,
                               double *R, long ldr, double *rnorm, double *xnorm, cudaStream_t s);
// (Xhi, Xlo) += s Z (or := s Z when assign), s = 2^ceil(log2 rnorm); znorm = max |s Z| (zeroed by the caller).
cudaError_t launch_update_dd(int n, int nrhs, const double *Z, long ldz, const double *rnorm, double *Xhi,
                             double *Xlo, long ldx, double *znorm, int assign, cudaStream_t s);
