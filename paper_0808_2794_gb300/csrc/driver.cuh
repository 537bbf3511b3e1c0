// driver.cuh -- internal entry of the solve driver (solver.cu).
#pragma once

#include "common.cuh"

// mp_gesv with an explicit choice of phase timing (timing creates CUDA events).
int mp_gesv_impl(int n, int nrhs, const double *dA, int lda, const double *dB, int ldb, double *dX,
                 int ldx, int32_t *dipiv, void *work, size_t work_bytes, const mp_opts *opts,
                 mp_stats *stats, void *stream, bool timing);
