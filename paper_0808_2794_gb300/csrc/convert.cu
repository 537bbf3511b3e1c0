// convert.cu -- W = fl(A) in the working precision with the norms the
// refinement needs (Section 2.1: "A is converted to single precision for the
// LU factorization ... the original A is kept"; DLANGE in Table 7).
//
// A (FP64, column-major, the caller's) is read once, coalesced, through a
// 64x64 shared-memory transpose into the row-major W; row sums of |a_ij| are
// accumulated for ||A||_inf, and any NaN/Inf raises MP_FLAG_NONFINITE_INPUT.
// Conversion to FP32 is round-to-nearest-even (fl32_rne: integer operations;
// the FP64 pipe is left to the row sums, one add per element).
#include "common.cuh"
#include "kernels.cuh"

namespace {

constexpr int kTile = 32;
constexpr int kColTiles = 4;  // each CTA walks 4 column tiles: fewer row-sum atomics

template <typename Tout>
__device__ __forceinline__ Tout cvt(double v);
template <> __device__ __forceinline__ float cvt<float>(double v) { return fl32_rne(v); }
template <> __device__ __forceinline__ double cvt<double>(double v) { return v; }

// 64 x 64 tiles: a warp reads 64 rows of a column as 16-byte pieces (512
// contiguous bytes per instruction), eight columns in flight per thread; after
// the transpose in shared memory a warp writes 64 values of a row (256 bytes
// of FP32) per instruction.  Long contiguous runs on both sides keep DRAM
// pages open; a CTA walks kColTiles column tiles to amortise the row-sum
// atomics.
constexpr int kT = 64;

template <typename Tout>
__global__ void __launch_bounds__(256)
convert_transpose_kernel(int n, const double *__restrict__ A, long lda, Tout *__restrict__ W,
                         long ldw, double *__restrict__ rowsum, MpDevStatus *st) {
    __shared__ Tout tile[kT][kT + 1];  // [column][row]
    __shared__ double rs[8][kT];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r0 = blockIdx.x * kT;
    const int ra = r0 + 2 * lane;  // this lane's two rows
    const bool vec = ((reinterpret_cast<uintptr_t>(A) | (uintptr_t)(lda * 8)) & 15) == 0;
    double rsum0 = 0.0, rsum1 = 0.0;
    bool bad = false;
    for (int ct = 0; ct < kColTiles; ++ct) {
        const int c0 = (blockIdx.y * kColTiles + ct) * kT;
        if (c0 >= n) break;
        double2 v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int c = c0 + warp + 8 * q;
            const double *src = A + (long)c * lda + ra;
            if (c < n && vec && ra + 1 < n) {
                v[q] = __ldcs(reinterpret_cast<const double2 *>(src));
            } else {
                v[q].x = (c < n && ra < n) ? __ldcs(src) : 0.0;
                v[q].y = (c < n && ra + 1 < n) ? __ldcs(src + 1) : 0.0;
            }
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            bad |= nonfinite_f64(v[q].x) | nonfinite_f64(v[q].y);
            rsum0 += fabs(v[q].x);
            rsum1 += fabs(v[q].y);
            tile[warp + 8 * q][2 * lane] = cvt<Tout>(v[q].x);
            tile[warp + 8 * q][2 * lane + 1] = cvt<Tout>(v[q].y);
        }
        __syncthreads();
        // rows r0 + warp + 8 q, columns c0 + 2 lane, c0 + 2 lane + 1
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int r = r0 + warp + 8 * q, c = c0 + 2 * lane;
            if (r < n) {
                Tout *dst = W + (long)r * ldw + c;
                const Tout x0 = tile[2 * lane][warp + 8 * q], x1 = tile[2 * lane + 1][warp + 8 * q];
                if (sizeof(Tout) == 4 && c + 1 < n && ((reinterpret_cast<uintptr_t>(dst) & 7) == 0)) {
                    float2 pr;
                    pr.x = (float)x0;
                    pr.y = (float)x1;
                    *reinterpret_cast<float2 *>(dst) = pr;
                } else {
                    if (c < n) dst[0] = x0;
                    if (c + 1 < n) dst[1] = x1;
                }
            }
        }
        __syncthreads();
    }
    if (bad) mp_flag(st, MP_FLAG_NONFINITE_INPUT);
    rs[warp][2 * lane] = rsum0;
    rs[warp][2 * lane + 1] = rsum1;
    __syncthreads();
    if (threadIdx.x < kT) {
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < 8; ++w) t += rs[w][threadIdx.x];
        if (r0 + threadIdx.x < n) atomicAdd(&rowsum[r0 + threadIdx.x], t);
    }
}

// Symmetric A given by its lower triangle: W[r][c] = fl(a_rc) for r >= c
// only (the upper triangle of A is not read and W's is not written).  Row
// sums of the full symmetric |A|: a strictly-lower a_rc counts for rows r
// and c.  Grid: one CTA per 32 x 32 tile, tiles above the diagonal exit.
template <typename Tout>
__global__ void __launch_bounds__(256)
convert_lower_kernel(int n, const double *__restrict__ A, long lda, Tout *__restrict__ W, long ldw,
                     double *__restrict__ rowsum, MpDevStatus *st) {
    __shared__ Tout tile[kTile][kTile + 1];
    __shared__ double rs[8][kTile];
    const int r0 = blockIdx.y * kTile, c0 = blockIdx.x * kTile;
    if (c0 > r0) return;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    double rsum = 0.0;
    bool bad = false;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int c = c0 + ty + 8 * q, r = r0 + tx;
        double v = 0.0;
        if (r < n && c <= r) v = A[(long)c * lda + r];
        bad |= nonfinite_f64(v);
        rsum += fabs(v);
        // strictly lower entries also count for row c: reduce over the 32 rows r
        double cs = (r > c) ? fabs(v) : 0.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) cs += __shfl_xor_sync(0xffffffffu, cs, off);
        if (tx == 0 && c < n && cs != 0.0) atomicAdd(&rowsum[c], cs);
        tile[ty + 8 * q][tx] = cvt<Tout>(v);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int r = r0 + ty + 8 * q, c = c0 + tx;
        if (r < n && c <= r) W[(long)r * ldw + c] = tile[tx][ty + 8 * q];
    }
    if (bad) mp_flag(st, MP_FLAG_NONFINITE_INPUT);
    rs[ty][tx] = rsum;
    __syncthreads();
    if (ty == 0) {
        double t = 0.0;
#pragma unroll
        for (int q = 0; q < 8; ++q) t += rs[q][tx];
        if (r0 + tx < n && t != 0.0) atomicAdd(&rowsum[r0 + tx], t);
    }
}

__global__ void __launch_bounds__(1024) max_reduce_kernel(int n, const double *__restrict__ v, double *out) {
    __shared__ double wm[32];
    double m = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double x = v[i];
        if (x > m || x != x) m = (x != x) ? __longlong_as_double(0x7ff0000000000000LL) : x;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? wm[threadIdx.x] : 0.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
        if (threadIdx.x == 0) *out = m;
    }
}

}  // namespace

template <typename Tout>
cudaError_t launch_convert_transpose(int n, const double *A, long lda, Tout *W, long ldw,
                                     double *rowsum, MpDevStatus *st, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    dim3 grid((n + kT - 1) / kT, (n + kT * kColTiles - 1) / (kT * kColTiles));
    mp_note_launch();
    convert_transpose_kernel<Tout><<<grid, 256, 0, s>>>(n, A, lda, W, ldw, rowsum, st);
    return cudaGetLastError();
}
template cudaError_t launch_convert_transpose<float>(int, const double *, long, float *, long,
                                                     double *, MpDevStatus *, cudaStream_t);
template cudaError_t launch_convert_transpose<double>(int, const double *, long, double *, long,
                                                      double *, MpDevStatus *, cudaStream_t);

template <typename Tout>
cudaError_t launch_convert_lower(int n, const double *A, long lda, Tout *W, long ldw, double *rowsum,
                                 MpDevStatus *st, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int nt = (n + kTile - 1) / kTile;
    mp_note_launch();
    convert_lower_kernel<Tout><<<dim3(nt, nt), dim3(32, 8), 0, s>>>(n, A, lda, W, ldw, rowsum, st);
    return cudaGetLastError();
}
template cudaError_t launch_convert_lower<float>(int, const double *, long, float *, long, double *,
                                                 MpDevStatus *, cudaStream_t);
template cudaError_t launch_convert_lower<double>(int, const double *, long, double *, long, double *,
                                                  MpDevStatus *, cudaStream_t);

cudaError_t launch_max_reduce(int n, const double *v, double *out, cudaStream_t s) {
    mp_note_launch();
    max_reduce_kernel<<<1, 1024, 0, s>>>(n, v, out);
    return cudaGetLastError();
}
