// tc_gemm.cuh -- tensor-core trailing update of the blocked factorization.
#pragma once

#include "common.cuh"

// Bytes of scratch the tensor-core update needs for order n, block width nb.
size_t tc_workspace_bytes(int n, int nb, int prec);

// A22[M x N] -= fl_p(L21[M x K]) * fl_p(U12[K x N]), all FP32 row-major,
// operands rounded to p = bf16 / fp16 (round to nearest even), products and
// sums in FP32 on the tensor cores (tcgen05, accumulators in TMEM).
// umax_pre (optional, device): max |U12| as the uint bits of a non-negative
// float (NaN counted as infinite), taken while U12 was formed; the scaled
// rungs then skip their own pass over U12.
cudaError_t tc_trailing_update(int prec, int M, int N, int K, const float *L21, long ldl,
                               const float *U12, long ldu, float *A22, long lda, void *ws,
                               MpDevStatus *st, cudaStream_t s, const unsigned *umax_pre = nullptr);

// C[M x N] -= fl_p(A[M x K]) fl_p(B[N x K])^T (B given row-major N x K, as for
// the symmetric update A22 -= L21 L21^T); lower != 0: only the tiles of C on
// or below its diagonal.
cudaError_t tc_update_nt(int prec, int M, int N, int K, const float *A, long lda, const float *B, long ldb,
                         float *C, long ldc, int lower, void *ws, MpDevStatus *st, cudaStream_t s);

// Standalone variant for tests/benchmarks: C[M x N] -= A[M x K] B[K x N].
cudaError_t tc_gemm_sub(int prec, int M, int N, int K, const float *A, long lda, const float *B,
                        long ldb, float *C, long ldc, void *ws, size_t ws_bytes, MpDevStatus *st,
                        cudaStream_t s);
