// dd.cu -- the residual and the update of iterative refinement with an
// extra-precise residual (Section 5: QDGESV, an FP64 factorization whose
// refinement computes the residual and keeps the solution in a precision
// beyond FP64).  Here the extended precision is double-double: a value is an
// unevaluated sum hi + lo of two doubles with |lo| <= ulp(hi)/2, carried by
// error-free transformations (Knuth's two-sum, the FMA two-product).
//
//   residual  r = b - A (x_hi + x_lo) per row: products A_ij x_hi,j split
//             exactly into p + e, the p summed with two-sum, every error term
//             and A_ij x_lo,j added into a compensation word; column chunks
//             over CTAs, partial (sum, compensation) pairs added in a fixed
//             order (deterministic); r is returned rounded to FP64 (the
//             right-hand side of the FP64 correction equation).
//   update    (x_hi, x_lo) += z, z in FP64: two-sum, then renormalised.
#include "common.cuh"
#include "kernels.cuh"

namespace {

constexpr int kRows = 256;
constexpr int kXs = 2048;  // x_hi and x_lo values of one chunk per CTA (32 KB)

__device__ __forceinline__ void two_sum(double a, double b, double &s, double &e) {
    s = a + b;
    const double bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void two_prod(double a, double b, double &p, double &e) {
    p = a * b;
    e = fma(a, b, -p);
}

// part_hi/part_lo[(ks * nrhs + c) * n + row] = sum and compensation of
// A[row, chunk ks] (x_hi + x_lo)[chunk ks, c], columns in order.
__global__ void __launch_bounds__(kRows)
residual_dd_partial_kernel(int n, int nrhs, const double *__restrict__ A, long lda, const double *__restrict__ Xhi,
                           const double *__restrict__ Xlo, long ldx, double *__restrict__ part_hi,
                           double *__restrict__ part_lo, int chunk) {
    __shared__ double xh[kXs / 2], xl[kXs / 2];
    const int row = blockIdx.x * kRows + threadIdx.x;
    const int ks = blockIdx.y, c = blockIdx.z;
    const int c0 = ks * chunk, len = max(0, min(n, c0 + chunk) - c0);
    for (int t = threadIdx.x; t < len; t += kRows) {
        xh[t] = Xhi[(long)c * ldx + c0 + t];
        xl[t] = Xlo[(long)c * ldx + c0 + t];
    }
    __syncthreads();
    if (row >= n) return;
    const double *a = A + (long)c0 * lda + row;
    double s = 0.0, comp = 0.0;
    int j = 0;
    for (; j + 8 <= len; j += 8) {  // 8 column loads in flight, products in column order
        double av[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) av[t] = __ldcs(a + (long)(j + t) * lda);
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            double p, ep, u, es;
            two_prod(av[t], xh[j + t], p, ep);
            two_sum(s, p, u, es);
            s = u;
            comp += ep + es;
            comp = fma(av[t], xl[j + t], comp);
        }
    }
    for (; j < len; ++j) {
        const double a0 = a[(long)j * lda];
        double p, ep, u, es;
        two_prod(a0, xh[j], p, ep);
        two_sum(s, p, u, es);
        s = u;
        comp += ep + es;
        comp = fma(a0, xl[j], comp);
    }
    part_hi[((long)ks * nrhs + c) * n + row] = s;
    part_lo[((long)ks * nrhs + c) * n + row] = comp;
}

// r = b - (sum of the partials), the partials added with two-sum in chunk
// order; R gets r rounded to FP64, rnorm/xnorm the max |r| and |x_hi|.
__global__ void __launch_bounds__(256)
residual_dd_finalize_kernel(int n, int nrhs, const double *__restrict__ part_hi, const double *__restrict__ part_lo,
                            int ksplit, const double *__restrict__ B, long ldb, const double *__restrict__ Xhi,
                            long ldx, double *__restrict__ R, long ldr, double *rnorm, double *xnorm) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    double rv = 0.0, xv = 0.0;
    if (row < n) {
        double s = 0.0, comp = 0.0;
        for (int ks = 0; ks < ksplit; ++ks) {
            double u, e;
            two_sum(s, part_hi[((long)ks * nrhs + c) * n + row], u, e);
            s = u;
            comp += e + part_lo[((long)ks * nrhs + c) * n + row];
        }
        double r, e;
        two_sum(B[(long)c * ldb + row], -s, r, e);  // b - (s + comp)
        r = r + (e - comp);
        R[(long)c * ldr + row] = r;
        rv = fabs(r);
        xv = fabs(Xhi[(long)c * ldx + row]);
        if (rv != rv) rv = __longlong_as_double(0x7ff0000000000000LL);
        if (xv != xv) xv = __longlong_as_double(0x7ff0000000000000LL);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        rv = fmax(rv, __shfl_xor_sync(0xffffffffu, rv, off));
        xv = fmax(xv, __shfl_xor_sync(0xffffffffu, xv, off));
    }
    if ((threadIdx.x & 31) == 0) {
        atomic_max_nonneg(&rnorm[c], rv);
        atomic_max_nonneg(&xnorm[c], xv);
    }
}

__device__ __forceinline__ double pow2_ceil_dd(double v) {
    if (!(v > 0.0) || !(v <= 1.79769313486231570815e308)) return 1.0;
    int e;
    const double m = frexp(v, &e);
    return (m == 0.5) ? ldexp(1.0, e - 1) : ldexp(1.0, e);
}

// (x_hi, x_lo) += s z (z the FP64 correction of the scaled right-hand side,
// s = 2^ceil(log2 rnorm)), or := s z when assign; znorm = max |s z|.
__global__ void __launch_bounds__(256)
update_dd_kernel(int n, const double *__restrict__ Z, long ldz, const double *__restrict__ rnorm, double *Xhi,
                 double *Xlo, long ldx, double *znorm, int assign) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    double zv = 0.0;
    if (row < n) {
        const double z = Z[(long)c * ldz + row] * pow2_ceil_dd(rnorm[c]);
        double *xh = Xhi + (long)c * ldx + row, *xl = Xlo + (long)c * ldx + row;
        if (assign) {
            *xh = z;
            *xl = 0.0;
        } else {
            double s, e;
            two_sum(*xh, z, s, e);
            e += *xl;
            const double h = s + e;  // renormalise: |lo| <= ulp(hi) / 2
            *xh = h;
            *xl = e - (h - s);
        }
        zv = fabs(z);
        if (zv != zv) zv = __longlong_as_double(0x7ff0000000000000LL);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) zv = fmax(zv, __shfl_xor_sync(0xffffffffu, zv, off));
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg(&znorm[c], zv);
}

}  // namespace

int residual_dd_ksplit(int n) {
    const int rowtiles = (n + kRows - 1) / kRows;
    int ks = (4 * 152 + rowtiles - 1) / rowtiles;
    const int max_by_len = (n + 63) / 64;
    if (ks > max_by_len) ks = max_by_len;
    if (ks < 1) ks = 1;
    while ((n + ks - 1) / ks > kXs / 2) ++ks;
    return ks;
}

cudaError_t launch_residual_dd(int n, int nrhs, const double *A, long lda, const double *Xhi, const double *Xlo,
                               long ldx, const double *B, long ldb, double *part_hi, double *part_lo, int ksplit,
                               double *R, long ldr, double *rnorm, double *xnorm, cudaStream_t s) {
    if (n <= 0 || nrhs <= 0) return cudaSuccess;
    const int chunk = (n + ksplit - 1) / ksplit;
    if (chunk > kXs / 2) return cudaErrorInvalidValue;
    mp_note_launch(2);
    residual_dd_partial_kernel<<<dim3((n + kRows - 1) / kRows, ksplit, nrhs), kRows, 0, s>>>(
        n, nrhs, A, lda, Xhi, Xlo, ldx, part_hi, part_lo, chunk);
    residual_dd_finalize_kernel<<<dim3((n + 255) / 256, nrhs), 256, 0, s>>>(n, nrhs, part_hi, part_lo, ksplit, B, ldb,
                                                                            Xhi, ldx, R, ldr, rnorm, xnorm);
    return cudaGetLastError();
}

cudaError_t launch_update_dd(int n, int nrhs, const double *Z, long ldz, const double *rnorm, double *Xhi,
                             double *Xlo, long ldx, double *znorm, int assign, cudaStream_t s) {
    if (n <= 0 || nrhs <= 0) return cudaSuccess;
    mp_note_launch();
    update_dd_kernel<<<dim3((n + 255) / 256, nrhs), 256, 0, s>>>(n, Z, ldz, rnorm, Xhi, Xlo, ldx, znorm, assign);
    return cudaGetLastError();
}
