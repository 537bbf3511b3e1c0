// batched.cuh -- internal interface of the batched small-system solver.
#pragma once

#include "common.cuh"

// Device description of one system of a batch (written by the host, the
// kernel fills iter/flags/info/bwd).
struct BatchSys {
    int n, nrhs, lda, ldb, ldx, ldw;
    const double *A, *B;
    double *X;
    int32_t *ipiv;
    void *W;      // n x ldw working matrix (FP32, or FP64 in the fallback pass)
    double *R;    // n x nrhs FP64 residual
    int *perm;    // composed row permutation
    void *Dinv;   // inverses of the 32 x 32 diagonal blocks of L and U
    int iter, info;
    unsigned flags;
    int nb;       // panel width of the low-precision factorization (from the schedule)
    double bwd;
};

// Workspace bytes for the batch (fp64: room for the FP64 fallback pass);
// per_sys_off (optional, batch entries) receives each system's W offset.
size_t batched_layout(int batch, const int *n, const int *nrhs, bool fp64, size_t *per_sys_off);

// Runs the batch (arguments validated by the caller).  Returns 0, or -1 with
// *cerr set when a CUDA call failed.
int batched_run(int batch, const int *n, const int *nrhs, const double *const *A, const int *lda,
                const double *const *B, const int *ldb, double *const *X, const int *ldx, int32_t *const *ipiv,
                int *iter, unsigned *flags, int *info, void *work, const mp_opts &o, cudaStream_t s,
                cudaError_t *cerr);
