// refine.cu -- the FP64 steps of the refinement loop (Algorithm 1, steps 4
// and 7 at eps_d; DGEMM residual and DAXPY update, Section 3.1.1).
//
// Residual R = B - A X with the caller's FP64 column-major A: each thread owns
// one row and walks a chunk of columns (coalesced: a warp reads 256 contiguous
// bytes of a column), the column chunks are split over CTAs, and the partial
// sums are added in a fixed order by the finalize kernel (deterministic).
// The arithmetic is FP64 FMA throughout.
#include "common.cuh"
#include "kernels.cuh"

namespace {

constexpr int kRows = 256;   // rows per CTA (one per thread)
constexpr int kMaxRhs = 8;
constexpr int kXsElems = 4096;  // 32 KB of x values per CTA

__device__ __forceinline__ double pow2_ceil(double v) {
    if (!(v > 0.0) || !(v <= 1.79769313486231570815e308)) return 1.0;
    int e;
    const double m = frexp(v, &e);
    return (m == 0.5) ? ldexp(1.0, e - 1) : ldexp(1.0, e);
}

template <int NR>
__global__ void __launch_bounds__(kRows)
residual_partial_kernel(int n, int nrhs, const double *__restrict__ A, long lda,
                        const double *__restrict__ X, long ldx, double *__restrict__ part,
                        int chunk) {
    __shared__ __align__(16) double xsf[kXsElems];  // chunk * NR <= kXsElems
    const int row = blockIdx.x * kRows + threadIdx.x;
    const int ks = blockIdx.y;
    const int c0 = ks * chunk;
    const int c1 = min(n, c0 + chunk);
    const int len = max(0, c1 - c0);
    for (int t = threadIdx.x; t < len * NR; t += blockDim.x) {
        const int j = t / NR, c = t % NR;
        xsf[t] = (c < nrhs) ? X[(long)c * ldx + c0 + j] : 0.0;
    }
    __syncthreads();
    if (row >= n) return;
    double acc[NR];
#pragma unroll
    for (int c = 0; c < NR; ++c) acc[c] = 0.0;
    const double *a = A + (long)c0 * lda + row;
    int j = 0;
    // 8 column loads in flight per thread (the products keep column order)
    for (; j + 8 <= len; j += 8) {
        double av[8], xv[8 * NR];
#pragma unroll
        for (int t = 0; t < 8; ++t) av[t] = __ldcs(a + (long)(j + t) * lda);
        // the 8 x NR values of these columns: 16-byte shared-memory loads
        // (j is a multiple of 8, so the first value is 16-byte aligned)
#pragma unroll
        for (int q = 0; q < 4 * NR; ++q) {
            const double2 v = reinterpret_cast<const double2 *>(xsf + j * NR)[q];
            xv[2 * q] = v.x;
            xv[2 * q + 1] = v.y;
        }
#pragma unroll
        for (int t = 0; t < 8; ++t)
#pragma unroll
            for (int c = 0; c < NR; ++c) acc[c] = fma(av[t], xv[t * NR + c], acc[c]);
    }
    for (; j < len; ++j) {
        const double a0 = a[(long)j * lda];
#pragma unroll
        for (int c = 0; c < NR; ++c) acc[c] = fma(a0, xsf[j * NR + c], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < NR; ++c)
        if (c < nrhs) part[((long)ks * nrhs + c) * n + row] = acc[c];
}

// Symmetric A from its lower triangle (the DSYMM step of the Cholesky
// variant, Section 3.1.1; half of A is read).  One CTA per 64 x 64 block
// (I, J), I >= J, of the lower triangle; it writes the contribution of
// block column J to the rows of block I (A_IJ x_J) and, for I > J, of block
// column I to the rows of block J (A_IJ^T x_I).  part[K][c][i] then holds,
// for every row i, the product of block column K of the full symmetric
// matrix with x, and the finalize kernel adds the K in order.
constexpr int kSymBS = 64;

__host__ __device__ constexpr size_t sym_smem_bytes(int nr) {
    return sizeof(double) * ((size_t)kSymBS * (kSymBS + 1) + 2 * (size_t)kSymBS * nr + 4 * (size_t)kSymBS * nr);
}

template <int NR>
__global__ void __launch_bounds__(256)
residual_sym_partial_kernel(int n, int nrhs, const double *__restrict__ A, long lda,
                            const double *__restrict__ X, long ldx, double *__restrict__ part) {
    extern __shared__ __align__(16) unsigned char raw[];
    double(*As)[kSymBS + 1] = reinterpret_cast<double(*)[kSymBS + 1]>(raw);  // As[col][row]
    double *xJ = reinterpret_cast<double *>(raw) + kSymBS * (kSymBS + 1);     // [64][NR]
    double *xI = xJ + kSymBS * NR;
    double *red = xI + kSymBS * NR;                                          // [4][64][NR]
    // block index -> (I, J), I >= J, t = I (I + 1) / 2 + J
    const long t = blockIdx.x;
    int I = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((long)I * (I + 1) / 2 > t) --I;
    while ((long)(I + 1) * (I + 2) / 2 <= t) ++I;
    const int J = (int)(t - (long)I * (I + 1) / 2);
    const int i0 = I * kSymBS, j0 = J * kSymBS;
    const int tid = threadIdx.x, lane64 = tid & 63, q = tid >> 6;
    for (int cc = q; cc < kSymBS; cc += 4) {
        const int gr = i0 + lane64, gc = j0 + cc;
        const bool in = gr < n && gc < n && (I != J || lane64 >= cc);
        As[cc][lane64] = in ? __ldcs(A + (long)gc * lda + gr) : 0.0;
    }
    for (int e = tid; e < kSymBS * NR; e += blockDim.x) {
        const int r = e / NR, c = e % NR;
        xJ[e] = (c < nrhs && j0 + r < n) ? X[(long)c * ldx + j0 + r] : 0.0;
        xI[e] = (c < nrhs && i0 + r < n) ? X[(long)c * ldx + i0 + r] : 0.0;
    }
    __syncthreads();
    // direct: rows of I, columns cc in [16q, 16q + 16)
    double acc[NR];
#pragma unroll
    for (int c = 0; c < NR; ++c) acc[c] = 0.0;
    for (int k = 0; k < 16; ++k) {
        const int cc = q * 16 + k;
        const double a = (I != J || cc <= lane64) ? As[cc][lane64] : As[lane64][cc];
#pragma unroll
        for (int c = 0; c < NR; ++c) acc[c] = fma(a, xJ[cc * NR + c], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < NR; ++c) red[(q * kSymBS + lane64) * NR + c] = acc[c];
    __syncthreads();
    if (tid < kSymBS && i0 + tid < n) {
#pragma unroll
        for (int c = 0; c < NR; ++c) {
            if (c >= nrhs) break;
            double sum = red[(0 * kSymBS + tid) * NR + c];
            sum += red[(1 * kSymBS + tid) * NR + c];
            sum += red[(2 * kSymBS + tid) * NR + c];
            sum += red[(3 * kSymBS + tid) * NR + c];
            part[((long)J * nrhs + c) * n + i0 + tid] = sum;
        }
    }
    if (I == J) return;
    __syncthreads();
    // transposed: columns cc = lane64 of J, rows in [16q, 16q + 16)
#pragma unroll
    for (int c = 0; c < NR; ++c) acc[c] = 0.0;
    for (int k = 0; k < 16; ++k) {
        const int rr = q * 16 + k;
        const double a = As[lane64][rr];
#pragma unroll
        for (int c = 0; c < NR; ++c) acc[c] = fma(a, xI[rr * NR + c], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < NR; ++c) red[(q * kSymBS + lane64) * NR + c] = acc[c];
    __syncthreads();
    if (tid < kSymBS && j0 + tid < n) {
#pragma unroll
        for (int c = 0; c < NR; ++c) {
            if (c >= nrhs) break;
            double sum = red[(0 * kSymBS + tid) * NR + c];
            sum += red[(1 * kSymBS + tid) * NR + c];
            sum += red[(2 * kSymBS + tid) * NR + c];
            sum += red[(3 * kSymBS + tid) * NR + c];
            part[((long)I * nrhs + c) * n + j0 + tid] = sum;
        }
    }
}

// Transposed residual for the adjoint solve: R = G - A^T L.  A CTA of 16
// warps takes 16 columns of A (rows of A^T); each warp reads its column
// coalesced, the matching chunk of L is staged in shared memory (c-major),
// and the lane partial sums are combined by a fixed shuffle tree.
constexpr int kTransWarps = 16;
constexpr int kTransChunk = 256;

template <int NR>
__global__ void __launch_bounds__(kTransWarps * 32)
residual_trans_kernel(int n, int nrhs, const double *__restrict__ A, long lda, const double *__restrict__ L,
                      long ldl, const double *__restrict__ G, long ldg, double *__restrict__ R, long ldr,
                      double *rnorm, double *xnorm, MpDevStatus *st) {
    __shared__ double ls[NR][kTransChunk];
    __shared__ double red_r[kTransWarps][NR], red_x[kTransWarps][NR];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int col = blockIdx.x * kTransWarps + warp;
    double acc[NR];
#pragma unroll
    for (int c = 0; c < NR; ++c) acc[c] = 0.0;
    const double *a = A + (long)min(col, n - 1) * lda;
    for (int j0 = 0; j0 < n; j0 += kTransChunk) {
        const int len = min(kTransChunk, n - j0);
        __syncthreads();
        for (int e = threadIdx.x; e < NR * kTransChunk; e += blockDim.x) {
            const int c = e / kTransChunk, j = e % kTransChunk;
            ls[c][j] = (c < nrhs && j < len) ? L[(long)c * ldl + j0 + j] : 0.0;
        }
        __syncthreads();
        if (col < n)
            for (int j = lane; j < len; j += 32) {
                const double av = __ldcs(a + j0 + j);
#pragma unroll
                for (int c = 0; c < NR; ++c) acc[c] = fma(av, ls[c][j], acc[c]);
            }
    }
#pragma unroll
    for (int c = 0; c < NR; ++c)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], off);
    if (lane == 0) {
#pragma unroll
        for (int c = 0; c < NR; ++c) {
            double rv = 0.0, xv = 0.0;
            if (col < n && c < nrhs) {
                const double r = G[(long)c * ldg + col] - acc[c];
                R[(long)c * ldr + col] = r;
                rv = fabs(r);
                xv = fabs(L[(long)c * ldl + col]);
                if (rv != rv) rv = __longlong_as_double(0x7ff0000000000000LL);
                if (xv != xv) xv = __longlong_as_double(0x7ff0000000000000LL);
            }
            red_r[warp][c] = rv;
            red_x[warp][c] = xv;
        }
    }
    __syncthreads();
    if (threadIdx.x < NR && threadIdx.x < nrhs) {
        double rv = 0.0, xv = 0.0;
        for (int w = 0; w < kTransWarps; ++w) {
            rv = fmax(rv, red_r[w][threadIdx.x]);
            xv = fmax(xv, red_x[w][threadIdx.x]);
        }
        atomic_max_nonneg(&rnorm[threadIdx.x], rv);
        atomic_max_nonneg(&xnorm[threadIdx.x], xv);
    }
    (void)st;
}

// Abar[i, j] = -sum_c L[i, c] X[j, c]; 64 x 64 tile per CTA, writes coalesced along i.
__global__ void __launch_bounds__(256)
outer_neg_kernel(int n, int nrhs, const double *__restrict__ L, long ldl, const double *__restrict__ X, long ldx,
                 double *__restrict__ Abar, long ldab) {
    __shared__ double lt[kMaxRhs][64], xt[kMaxRhs][64];
    const int i0 = blockIdx.x * 64, j0 = blockIdx.y * 64;
    for (int e = threadIdx.x; e < kMaxRhs * 64; e += blockDim.x) {
        const int c = e / 64, r = e % 64;
        lt[c][r] = (c < nrhs && i0 + r < n) ? L[(long)c * ldl + i0 + r] : 0.0;
        xt[c][r] = (c < nrhs && j0 + r < n) ? X[(long)c * ldx + j0 + r] : 0.0;
    }
    __syncthreads();
    const int i = threadIdx.x & 63, jg = threadIdx.x >> 6;
    if (i0 + i >= n) return;
    for (int k = 0; k < 16; ++k) {
        const int j = jg * 16 + k;
        if (j0 + j >= n) break;
        double v = 0.0;
        for (int c = 0; c < nrhs; ++c) v = fma(lt[c][i], xt[c][j], v);
        Abar[(long)(j0 + j) * ldab + i0 + i] = -v;
    }
}

__global__ void __launch_bounds__(256)
residual_finalize_kernel(int n, int nrhs, const double *__restrict__ part, int ksplit,
                         const double *__restrict__ B, long ldb, const double *__restrict__ X,
                         long ldx, double *__restrict__ R, long ldr, double *rnorm, double *xnorm,
                         MpDevStatus *st) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    double rv = 0.0, xv = 0.0;
    if (row < n) {
        double s = 0.0;
        for (int ks = 0; ks < ksplit; ++ks) s += part[((long)ks * nrhs + c) * n + row];
        const double r = B ? B[(long)c * ldb + row] - s : s;  // B == nullptr: R = A X
        R[(long)c * ldr + row] = r;
        rv = fabs(r);
        xv = fabs(X[(long)c * ldx + row]);
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

template <typename T>
__global__ void __launch_bounds__(256)
update_kernel(int n, const T *__restrict__ Z, long ldz, const double *__restrict__ rnorm,
              double *__restrict__ X, long ldx, double *znorm, int assign, const int *__restrict__ scatter) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    double zv = 0.0;
    if (row < n) {
        const double s = pow2_ceil(rnorm[c]);
        const double z = (double)Z[(long)c * ldz + row] * s;
        double *x = X + (long)c * ldx + (scatter ? scatter[row] : row);
        *x = assign ? z : (*x + z);
        zv = fabs(z);
        if (zv != zv) zv = __longlong_as_double(0x7ff0000000000000LL);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) zv = fmax(zv, __shfl_xor_sync(0xffffffffu, zv, off));
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg(&znorm[c], zv);
}

__global__ void __launch_bounds__(256)
col_absmax_kernel(int n, const double *__restrict__ B, long ldb, double *out, MpDevStatus *st) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    double v = 0.0;
    if (row < n) {
        v = fabs(B[(long)c * ldb + row]);
        if (!(v <= 1.79769313486231570815e308)) {
            mp_flag(st, MP_FLAG_NONFINITE_INPUT);
            v = __longlong_as_double(0x7ff0000000000000LL);
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg(&out[c], v);
}

}  // namespace

static int rhs_pad(int nrhs) { return nrhs <= 1 ? 1 : nrhs <= 2 ? 2 : nrhs <= 4 ? 4 : 8; }

int residual_ksplit(int n, int nrhs) {
    const int rowtiles = (n + kRows - 1) / kRows;
    int ks = (4 * 152 + rowtiles - 1) / rowtiles;  // about four CTAs per SM
    const int max_by_len = (n + 63) / 64;          // keep chunks >= 64 columns
    if (ks > max_by_len) ks = max_by_len;
    if (ks < 1) ks = 1;
    const int cmax = kXsElems / rhs_pad(nrhs);
    while ((n + ks - 1) / ks > cmax) ++ks;         // chunk must fit shared memory
    return ks;
}

cudaError_t launch_residual_partial(int n, int nrhs, const double *A, long lda, const double *X,
                                    long ldx, double *part, int ksplit, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if (nrhs > kMaxRhs) return cudaErrorInvalidValue;
    const int chunk = (n + ksplit - 1) / ksplit;
    if (chunk * rhs_pad(nrhs) > kXsElems) return cudaErrorInvalidValue;
    dim3 grid((n + kRows - 1) / kRows, ksplit);
    mp_note_launch();
    if (nrhs <= 1)
        residual_partial_kernel<1><<<grid, kRows, 0, s>>>(n, nrhs, A, lda, X, ldx, part, chunk);
    else if (nrhs <= 2)
        residual_partial_kernel<2><<<grid, kRows, 0, s>>>(n, nrhs, A, lda, X, ldx, part, chunk);
    else if (nrhs <= 4)
        residual_partial_kernel<4><<<grid, kRows, 0, s>>>(n, nrhs, A, lda, X, ldx, part, chunk);
    else
        residual_partial_kernel<8><<<grid, kRows, 0, s>>>(n, nrhs, A, lda, X, ldx, part, chunk);
    return cudaGetLastError();
}

int residual_sym_blocks(int n) { return (n + kSymBS - 1) / kSymBS; }

cudaError_t launch_residual_sym_partial(int n, int nrhs, const double *A, long lda, const double *X, long ldx,
                                        double *part, cudaStream_t s) {
    if (n <= 0 || nrhs <= 0) return cudaSuccess;
    if (nrhs > kMaxRhs) return cudaErrorInvalidValue;
    const long nb = residual_sym_blocks(n);
    const long grid = nb * (nb + 1) / 2;
    const int nr = rhs_pad(nrhs);
    const size_t smem = sym_smem_bytes(nr);
    cudaError_t e = cudaSuccess;
    mp_note_launch();
#define MP_SYM_LAUNCH(NRV)                                                                                     \
    e = cudaFuncSetAttribute(residual_sym_partial_kernel<NRV>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             (int)smem);                                                                   \
    if (e != cudaSuccess) return e;                                                                        \
    residual_sym_partial_kernel<NRV><<<(unsigned)grid, 256, smem, s>>>(n, nrhs, A, lda, X, ldx, part);
    if (nr == 1) { MP_SYM_LAUNCH(1) }
    else if (nr == 2) { MP_SYM_LAUNCH(2) }
    else if (nr == 4) { MP_SYM_LAUNCH(4) }
    else { MP_SYM_LAUNCH(8) }
#undef MP_SYM_LAUNCH
    return cudaGetLastError();
}

cudaError_t launch_residual_trans(int n, int nrhs, const double *A, long lda, const double *L, long ldl,
                                  const double *G, long ldg, double *R, long ldr, double *rnorm, double *xnorm,
                                  MpDevStatus *st, cudaStream_t s) {
    if (n <= 0 || nrhs <= 0) return cudaSuccess;
    if (nrhs > kMaxRhs) return cudaErrorInvalidValue;
    const int grid = (n + kTransWarps - 1) / kTransWarps;
    const int nr = rhs_pad(nrhs);
    mp_note_launch();
    if (nr == 1)
        residual_trans_kernel<1><<<grid, kTransWarps * 32, 0, s>>>(n, nrhs, A, lda, L, ldl, G, ldg, R, ldr, rnorm, xnorm, st);
    else if (nr == 2)
        residual_trans_kernel<2><<<grid, kTransWarps * 32, 0, s>>>(n, nrhs, A, lda, L, ldl, G, ldg, R, ldr, rnorm, xnorm, st);
    else if (nr == 4)
        residual_trans_kernel<4><<<grid, kTransWarps * 32, 0, s>>>(n, nrhs, A, lda, L, ldl, G, ldg, R, ldr, rnorm, xnorm, st);
    else
        residual_trans_kernel<8><<<grid, kTransWarps * 32, 0, s>>>(n, nrhs, A, lda, L, ldl, G, ldg, R, ldr, rnorm, xnorm, st);
    return cudaGetLastError();
}

cudaError_t launch_outer_neg(int n, int nrhs, const double *L, long ldl, const double *X, long ldx, double *Abar,
                             long ldab, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if (nrhs > kMaxRhs) return cudaErrorInvalidValue;
    dim3 grid((n + 63) / 64, (n + 63) / 64);
    mp_note_launch();
    outer_neg_kernel<<<grid, 256, 0, s>>>(n, nrhs, L, ldl, X, ldx, Abar, ldab);
    return cudaGetLastError();
}

cudaError_t launch_residual_finalize(int n, int nrhs, const double *part, int ksplit, const double *B,
                                     long ldb, const double *X, long ldx, double *R, long ldr,
                                     double *rnorm, double *xnorm, MpDevStatus *st, cudaStream_t s) {
    if (n <= 0 || nrhs <= 0) return cudaSuccess;
    dim3 grid((n + 255) / 256, nrhs);
    mp_note_launch();
    residual_finalize_kernel<<<grid, 256, 0, s>>>(n, nrhs, part, ksplit, B, ldb, X, ldx, R, ldr,
                                                  rnorm, xnorm, st);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_update(int n, int nrhs, const T *Z, long ldz, const double *rnorm, double *X,
                          long ldx, double *znorm, int assign, cudaStream_t s, const int *scatter) {
    if (n <= 0 || nrhs <= 0) return cudaSuccess;
    dim3 grid((n + 255) / 256, nrhs);
    mp_note_launch();
    update_kernel<T><<<grid, 256, 0, s>>>(n, Z, ldz, rnorm, X, ldx, znorm, assign, scatter);
    return cudaGetLastError();
}
template cudaError_t launch_update<float>(int, int, const float *, long, const double *, double *, long,
                                          double *, int, cudaStream_t, const int *);
template cudaError_t launch_update<double>(int, int, const double *, long, const double *, double *,
                                           long, double *, int, cudaStream_t, const int *);

cudaError_t launch_col_absmax(int n, int nrhs, const double *B, long ldb, double *out,
                              MpDevStatus *st, cudaStream_t s) {
    if (n <= 0 || nrhs <= 0) return cudaSuccess;
    dim3 grid((n + 255) / 256, nrhs);
    mp_note_launch();
    col_absmax_kernel<<<grid, 256, 0, s>>>(n, B, ldb, out, st);
    return cudaGetLastError();
}

// ============================================================================
// Building blocks of GMRES-based refinement (Section 2.2: a Krylov method on
// A d = r, right-preconditioned by M = (LU)^{-1} P; Section 4): FP64 dot
// products against the Krylov basis, projection, 2-norms, and the correction
// x += Z y.  Deterministic: every reduction has a fixed order.
// ============================================================================
namespace {

// out[j] = sum_i V[i, j] w[i] for j < k; one CTA per column.
__global__ void __launch_bounds__(1024)
dots_kernel(int n, const double *__restrict__ V, long ldv, const double *__restrict__ w, double *out) {
    __shared__ double red[32];
    const int j = blockIdx.x;
    const double *v = V + (long)j * ldv;
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s = fma(v[i], w[i], s);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (threadIdx.x == 0) out[j] = s;
    }
}

// w[i] -= sum_{j<k} V[i, j] h[j]
__global__ void __launch_bounds__(256)
project_kernel(int n, int k, const double *__restrict__ V, long ldv, const double *__restrict__ h, double *w) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = w[i];
    for (int j = 0; j < k; ++j) s = fma(-V[(long)j * ldv + i], h[j], s);
    w[i] = s;
}

// x[i] += sum_{j<k} Z[i, j] y[j]; znorm = max |sum| (atomic, zeroed first)
__global__ void __launch_bounds__(256)
correct_kernel(int n, int k, const double *__restrict__ Z, long ldz, const double *__restrict__ y, double *x,
               double *znorm) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double d = 0.0;
    if (i < n) {
        for (int j = 0; j < k; ++j) d = fma(Z[(long)j * ldz + i], y[j], d);
        x[i] += d;
    }
    double a = fabs(d);
    if (a != a) a = __longlong_as_double(0x7ff0000000000000LL);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) a = fmax(a, __shfl_xor_sync(0xffffffffu, a, off));
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg(znorm, a);
}

// dst = src / d
__global__ void __launch_bounds__(256)
scale_kernel(int n, const double *src, double d, double *dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[i] / d;
}

}  // namespace

cudaError_t launch_dots(int n, int k, const double *V, long ldv, const double *w, double *out, cudaStream_t s) {
    if (k <= 0) return cudaSuccess;
    mp_note_launch();
    dots_kernel<<<k, 1024, 0, s>>>(n, V, ldv, w, out);
    return cudaGetLastError();
}
cudaError_t launch_project(int n, int k, const double *V, long ldv, const double *h, double *w, cudaStream_t s) {
    if (k <= 0 || n <= 0) return cudaSuccess;
    mp_note_launch();
    project_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, k, V, ldv, h, w);
    return cudaGetLastError();
}
cudaError_t launch_correct(int n, int k, const double *Z, long ldz, const double *y, double *x, double *znorm,
                           cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    mp_note_launch();
    correct_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, k, Z, ldz, y, x, znorm);
    return cudaGetLastError();
}
cudaError_t launch_scale(int n, const double *src, double d, double *dst, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    mp_note_launch();
    scale_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, src, d, dst);
    return cudaGetLastError();
}
