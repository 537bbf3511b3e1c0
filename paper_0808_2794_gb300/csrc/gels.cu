// gels.cu -- linear least squares min ||b - A x||_2 (A m x n, m >= n, full
// column rank) by mixed-precision refinement of the augmented system
// (Section 6 names least squares among the algorithms the approach extends
// to; the augmented formulation is Bjorck's):
//
//     [ alpha I   A ] [ r / alpha ]   [ b ]
//     [ A^T       0 ] [ x         ] = [ 0 ]
//
// whose solution gives x and the residual r = b - A x.  The (m + n)-order
// matrix is built here and solved by the general driver (low-precision LU
// with partial pivoting, FP64 residual and refinement).  alpha is a power of
// two near ||A||_F / sqrt(8 n): for a well-conditioned A that is within a
// small factor of the smallest singular value over sqrt(2), where the
// augmented matrix's condition number is about 2 kappa_2(A) (a larger alpha
// grows it towards kappa_2(A)^2).
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "driver.cuh"
#include "kernels.cuh"

namespace {

// K = [alpha I, A; A^T, 0] (N = m + n, column-major, ldk); one thread per row
// of a column, columns over the grid's y dimension.
__global__ void __launch_bounds__(256)
build_augmented_kernel(int m, int n, const double *__restrict__ A, long lda, double alpha, double *__restrict__ K,
                       long ldk) {
    const int N = m + n;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    for (int j = blockIdx.y; j < N; j += gridDim.y) {
        if (i >= N) continue;
        double v = 0.0;
        if (j < m) v = i < m ? (i == j ? alpha : 0.0) : A[(long)(i - m) * lda + j];  // A^T below
        else if (i < m) v = A[(long)(j - m) * lda + i];
        K[(long)j * ldk + i] = v;
    }
}

// rhs = [B; 0]
__global__ void __launch_bounds__(256)
augmented_rhs_kernel(int m, int n, const double *__restrict__ B, long ldb, double *__restrict__ F, long ldf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, c = blockIdx.y;
    if (i < m + n) F[(long)c * ldf + i] = i < m ? B[(long)c * ldb + i] : 0.0;
}

// X = Y[m:, :], R = alpha Y[:m, :] (exact: alpha is a power of two)
__global__ void __launch_bounds__(256)
split_solution_kernel(int m, int n, const double *__restrict__ Y, long ldy, double alpha, double *__restrict__ X,
                      long ldx, double *__restrict__ R, long ldr) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, c = blockIdx.y;
    if (i >= m + n) return;
    const double y = Y[(long)c * ldy + i];
    if (i >= m) X[(long)c * ldx + (i - m)] = y;
    else if (R) R[(long)c * ldr + i] = alpha * y;
}

// sum of squares of A (one atomic per block)
__global__ void __launch_bounds__(256)
sumsq_kernel(int m, int n, const double *__restrict__ A, long lda, double *out) {
    double s = 0.0;
    const long total = (long)m * n;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const double v = A[(e / m) * lda + e % m];
        s += v * v;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

struct GelsLayout {
    size_t K, F, Y, piv, nrm, solve, total;
};
GelsLayout gels_layout(int m, int n, int nrhs, const mp_opts *opts) {
    const size_t N = (size_t)m + n, r = (size_t)(nrhs > 0 ? nrhs : 1);
    auto al = [](size_t v) { return (v + 255) / 256 * 256; };
    GelsLayout L{};
    size_t off = 0;
    L.K = off; off += al(N * N * sizeof(double));
    L.F = off; off += al(N * r * sizeof(double));
    L.Y = off; off += al(N * r * sizeof(double));
    L.piv = off; off += al(N * sizeof(int32_t));
    L.nrm = off; off += 256;
    L.solve = off; off += al(mp_gesv_workspace_bytes((int)N, nrhs, opts));
    L.total = off;
    return L;
}

}  // namespace

extern "C" size_t mp_gels_workspace_bytes(int m, int n, int nrhs, const mp_opts *opts) {
    if (m < 0 || n < 0 || nrhs < 0 || (long)m + n > 65536) return 0;
    return gels_layout(m, n, nrhs, opts).total;
}

extern "C" int mp_gels(int m, int n, int nrhs, const double *dA, int lda, const double *dB, int ldb, double *dX,
                       int ldx, double *dR, int ldr, double alpha, void *work, size_t work_bytes, const mp_opts *opts,
                       mp_stats *stats, void *stream) {
    mp_set_error("");
    if (m < 0) return mp_arg_fail(1, "m < 0");
    if (n < 0 || n > m) return mp_arg_fail(2, "n must be in [0, m]");
    if ((long)m + n > 65536) return mp_arg_fail(1, "m + n > 65536 is not supported");
    if (nrhs < 0 || nrhs > 8) return mp_arg_fail(3, "nrhs must be in [0, 8]");
    if (m > 0 && n > 0 && !dA) return mp_arg_fail(4, "A is NULL");
    if (lda < (m > 1 ? m : 1)) return mp_arg_fail(5, "lda < max(1, m)");
    if (m > 0 && nrhs > 0 && !dB) return mp_arg_fail(6, "B is NULL");
    if (ldb < (m > 1 ? m : 1)) return mp_arg_fail(7, "ldb < max(1, m)");
    if (n > 0 && nrhs > 0 && !dX) return mp_arg_fail(8, "X is NULL");
    if (ldx < (n > 1 ? n : 1)) return mp_arg_fail(9, "ldx < max(1, n)");
    if (dR && ldr < (m > 1 ? m : 1)) return mp_arg_fail(11, "ldr < max(1, m)");
    if (!(alpha >= 0.0) || !std::isfinite(alpha)) return mp_arg_fail(12, "alpha must be >= 0 and finite");
    if (stats) std::memset(stats, 0, sizeof(*stats));
    if (m == 0 || n == 0 || nrhs == 0) return 0;
    const GelsLayout L = gels_layout(m, n, nrhs, opts);
    if (!work) return mp_arg_fail(13, "workspace is NULL");
    if (work_bytes < L.total) return mp_arg_fail(14, "workspace too small");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char *w = static_cast<char *>(work);
    const int N = m + n;
    double *K = reinterpret_cast<double *>(w + L.K), *F = reinterpret_cast<double *>(w + L.F);
    double *Y = reinterpret_cast<double *>(w + L.Y), *nrm = reinterpret_cast<double *>(w + L.nrm);
    if (alpha == 0.0) {  // the power of two nearest ||A||_F / sqrt(8 n)
        MP_CUDA_TRY(cudaMemsetAsync(nrm, 0, sizeof(double), s));
        mp_note_launch();
        sumsq_kernel<<<1216, 256, 0, s>>>(m, n, dA, lda, nrm);
        MP_CUDA_TRY(cudaGetLastError());
        double h = 0.0;
        MP_CUDA_TRY(cudaMemcpyAsync(&h, nrm, sizeof h, cudaMemcpyDeviceToHost, s));
        MP_CUDA_TRY(cudaStreamSynchronize(s));
        const double t = std::sqrt(h / (8.0 * n));
        alpha = (t > 0.0 && std::isfinite(t)) ? std::ldexp(1.0, (int)std::lround(std::log2(t))) : 1.0;
    }
    mp_note_launch(2);
    build_augmented_kernel<<<dim3((N + 255) / 256, N < 4096 ? N : 4096), 256, 0, s>>>(m, n, dA, lda, alpha, K, N);
    augmented_rhs_kernel<<<dim3((N + 255) / 256, nrhs), 256, 0, s>>>(m, n, dB, ldb, F, N);
    MP_CUDA_TRY(cudaGetLastError());
    const int r = mp_gesv(N, nrhs, K, N, F, N, Y, N, reinterpret_cast<int32_t *>(w + L.piv), w + L.solve,
                          work_bytes - L.solve, opts, stats, stream);
    if (r != 0) return r < 0 && r > -1000 ? mp_arg_fail(15, "augmented solve rejected the options") : r;
    mp_note_launch();
    split_solution_kernel<<<dim3((N + 255) / 256, nrhs), 256, 0, s>>>(m, n, Y, N, alpha, dX, ldx, dR, ldr);
    MP_CUDA_TRY(cudaGetLastError());
    MP_CUDA_TRY(cudaStreamSynchronize(s));
    return 0;
}
