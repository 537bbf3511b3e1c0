// trsv.cu -- triangular solves with the low-precision factors,
// L y = P r and U z = y (Algorithm 1 steps 2-3 and 5-6; SGETRS, Section
// 3.1.1).
//
// GB300 design: the factors are row-major, so every block row of L (or U)
// is a set of contiguous row segments.  The n rows are cut into 64-row
// blocks; the diagonal blocks are inverted once after the factorization, so
// that a block's own solve is a small parallel matrix-vector product.  One
// CTA per block row streams the off-diagonal blocks of its rows and
// subtracts their contribution as soon as the producing block is published
// (a per-block flag, "sync-free" wavefront).  CTAs take their block index
// from an atomic ticket, so a CTA only ever waits on CTAs that are already
// running; every wait is bounded and reports MP_FLAG_TIMEOUT if it gives up.
//
// The right-hand side r (FP64) is scaled by s = 2^ceil(log2 ||r||inf) before
// it is rounded to the working precision (exact power-of-two scaling keeps
// tiny late residuals out of the subnormal range).
#include "common.cuh"
#include "kernels.cuh"

namespace {

constexpr int BS = TRSV_BS;
constexpr int kMaxRhs = 8;

__device__ __forceinline__ double pow2_ceil(double v) {
    if (!(v > 0.0) || !(v <= 1.79769313486231570815e308)) return 1.0;
    int e;
    const double m = frexp(v, &e);
    return (m == 0.5) ? ldexp(1.0, e - 1) : ldexp(1.0, e);
}

// ---- inverses of the diagonal blocks ---------------------------------------
template <typename T>
__global__ void __launch_bounds__(BS)
diag_inverse_kernel(int n, const T *__restrict__ W, long ldw, T *__restrict__ Linv, T *__restrict__ Uinv) {
    __shared__ T blk[BS][BS + 1];
    __shared__ T x[BS][BS + 1];  // x[i][c]: column c of the inverse (thread c)
    const int b = blockIdx.x, c = threadIdx.x;
    const int r0 = b * BS;
    const int bs = min(BS, n - r0);
    for (int i = 0; i < BS; ++i) {
        const bool in = (i < bs) && (c < bs);
        blk[i][c] = in ? W[(long)(r0 + i) * ldw + r0 + c] : T(i == c ? 1 : 0);
    }
    __syncthreads();
    // unit lower: x_i = delta_ic - sum_{l<i} L_il x_l
    for (int i = 0; i < BS; ++i) {
        T s = T(i == c ? 1 : 0);
        for (int l = 0; l < i; ++l) s = fma(-blk[i][l], x[l][c], s);
        x[i][c] = s;
    }
    T *Lo = Linv + (long)b * BS * BS;
    for (int i = 0; i < BS; ++i) Lo[i * BS + c] = x[i][c];
    __syncthreads();
    // upper: x_i = (delta_ic - sum_{l>i} U_il x_l) / U_ii
    for (int i = BS - 1; i >= 0; --i) {
        T s = T(i == c ? 1 : 0);
        for (int l = i + 1; l < BS; ++l) s = fma(-blk[i][l], x[l][c], s);
        x[i][c] = s / blk[i][i];
    }
    T *Uo = Uinv + (long)b * BS * BS;
    for (int i = 0; i < BS; ++i) Uo[i * BS + c] = x[i][c];
}

// Waits (thread 0) until flags[j] >= epoch for the next dependency j, scanning
// ahead over already-published blocks; returns the first index not yet known
// to be ready after j (exclusive bound, in the direction of `step`).
__device__ __forceinline__ int advance_ready(const int *flags, int j, int stop, int step, int epoch,
                                             MpDevStatus *st, bool *ok) {
    const volatile int *vf = flags;
    if (!wait_flag_geq(vf + j, epoch, st, 1)) { *ok = false; return stop; }
    int q = j + step;
    while (q != stop && vf[q] >= epoch) q += step;
    __threadfence();
    return q;
}

// One CTA per 64-row block: thread (r = tid/4, seg = tid%4) owns row r and
// the 16-column segment seg of every 64-column block.
template <typename T, bool LOWER>
__global__ void __launch_bounds__(256)
trsv_block_kernel(int n, int nrhs, const T *__restrict__ W, long ldw, const T *__restrict__ Dinv,
                  const double *__restrict__ R, long ldr, const int *__restrict__ perm,
                  const double *__restrict__ rnorm, const T *__restrict__ Yin, long ldyin,
                  T *__restrict__ Yout, long ldyout, int *flags, int *ticket, int epoch,
                  MpDevStatus *st) {
    __shared__ int s_blk, s_ready;
    __shared__ bool s_ok;
    __shared__ T accs[kMaxRhs][BS];
    const int tid = threadIdx.x;
    const int r = tid >> 2, seg = tid & 3;
    const int nblk = (n + BS - 1) / BS;
    if (tid == 0) {
        const int t = atomicAdd(ticket, 1) - (epoch - 1) * nblk;
        s_blk = LOWER ? t : (nblk - 1 - t);
        s_ok = true;
    }
    __syncthreads();
    const int i = s_blk;
    if (i < 0 || i >= nblk) return;  // cannot happen with a correct ticket base
    const int row = i * BS + r;
    const bool rvalid = row < n;
    T part[kMaxRhs];
#pragma unroll
    for (int c = 0; c < kMaxRhs; ++c) part[c] = T(0);

    // dependencies: lower -> j = 0 .. i-1; upper -> j = nblk-1 .. i+1
    const int jstart = LOWER ? 0 : nblk - 1;
    const int jstop = LOWER ? i : i;
    const int step = LOWER ? 1 : -1;
    int ready = jstart;  // first dependency not yet known ready
    for (int j = jstart; j != jstop; j += step) {
        if (j == ready) {
            if (tid == 0) {
                bool ok = true;
                s_ready = advance_ready(flags, j, jstop, step, epoch, st, &ok);
                if (!ok) s_ok = false;
            }
            __syncthreads();
            if (!s_ok) return;  // timeout: flags already record it
            ready = s_ready;
        }
        if (rvalid) {
            const int c0 = j * BS + seg * 16;
            const T *wrow = W + (long)row * ldw + c0;
            T wv[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) wv[q] = (c0 + q < n) ? wrow[q] : T(0);
#pragma unroll
            for (int c = 0; c < kMaxRhs; ++c) {
                if (c < nrhs) {
                    const T *y = Yout + (long)c * ldyout + c0;
                    T acc = part[c];
#pragma unroll
                    for (int q = 0; q < 16; ++q)
                        if (c0 + q < n) acc = fma(wv[q], __ldcg(y + q), acc);
                    part[c] = acc;
                }
            }
        }
    }
    // reduce the four segment partials of each row
#pragma unroll
    for (int c = 0; c < kMaxRhs; ++c) {
        part[c] += __shfl_xor_sync(0xffffffffu, part[c], 1);
        part[c] += __shfl_xor_sync(0xffffffffu, part[c], 2);
    }
    if (seg == 0) {
#pragma unroll
        for (int c = 0; c < kMaxRhs; ++c) {
            if (c >= nrhs) break;
            T rhs = T(0);
            if (rvalid) {
                if (LOWER) {
                    const double s = pow2_ceil(rnorm[c]);
                    rhs = (T)(R[(long)c * ldr + perm[row]] / s);
                } else {
                    rhs = Yin[(long)c * ldyin + row];
                }
            }
            accs[c][r] = rvalid ? rhs - part[c] : T(0);
        }
    }
    __syncthreads();
    // y_i = Dinv_i * acc
    const T *D = Dinv + (long)i * BS * BS + r * BS + seg * 16;
    T dv[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) dv[q] = D[q];
    for (int c = 0; c < nrhs; ++c) {
        T acc = T(0);
#pragma unroll
        for (int q = 0; q < 16; ++q) acc = fma(dv[q], accs[c][seg * 16 + q], acc);
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        acc += __shfl_xor_sync(0xffffffffu, acc, 2);
        if (seg == 0 && rvalid) Yout[(long)c * ldyout + row] = acc;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) atomicExch(&flags[i], epoch);
}

}  // namespace

template <typename T>
cudaError_t launch_diag_inverses(int n, const T *W, long ldw, T *Linv, T *Uinv, cudaStream_t s) {
    const int nblk = (n + BS - 1) / BS;
    if (nblk == 0) return cudaSuccess;
    mp_note_launch();
    diag_inverse_kernel<T><<<nblk, BS, 0, s>>>(n, W, ldw, Linv, Uinv);
    return cudaGetLastError();
}
template cudaError_t launch_diag_inverses<float>(int, const float *, long, float *, float *, cudaStream_t);
template cudaError_t launch_diag_inverses<double>(int, const double *, long, double *, double *, cudaStream_t);

template <typename T>
cudaError_t launch_trsv_lower(int n, int nrhs, const T *W, long ldw, const T *Linv, const double *R,
                              long ldr, const int *perm, const double *rnorm, T *Y, long ldy,
                              int *flags, int *ticket, int epoch, MpDevStatus *st, cudaStream_t s) {
    if (nrhs > kMaxRhs) return cudaErrorInvalidValue;
    const int nblk = (n + BS - 1) / BS;
    if (nblk == 0) return cudaSuccess;
    mp_note_launch();
    trsv_block_kernel<T, true><<<nblk, 256, 0, s>>>(n, nrhs, W, ldw, Linv, R, ldr, perm, rnorm,
                                                    nullptr, 0, Y, ldy, flags, ticket, epoch, st);
    return cudaGetLastError();
}
template cudaError_t launch_trsv_lower<float>(int, int, const float *, long, const float *, const double *,
                                              long, const int *, const double *, float *, long, int *,
                                              int *, int, MpDevStatus *, cudaStream_t);
template cudaError_t launch_trsv_lower<double>(int, int, const double *, long, const double *,
                                               const double *, long, const int *, const double *,
                                               double *, long, int *, int *, int, MpDevStatus *,
                                               cudaStream_t);

template <typename T>
cudaError_t launch_trsv_upper(int n, int nrhs, const T *W, long ldw, const T *Uinv, const T *Y,
                              long ldy, T *Z, long ldz, int *flags, int *ticket, int epoch,
                              MpDevStatus *st, cudaStream_t s) {
    if (nrhs > kMaxRhs) return cudaErrorInvalidValue;
    const int nblk = (n + BS - 1) / BS;
    if (nblk == 0) return cudaSuccess;
    mp_note_launch();
    trsv_block_kernel<T, false><<<nblk, 256, 0, s>>>(n, nrhs, W, ldw, Uinv, nullptr, 0, nullptr,
                                                     nullptr, Y, ldy, Z, ldz, flags, ticket, epoch, st);
    return cudaGetLastError();
}
template cudaError_t launch_trsv_upper<float>(int, int, const float *, long, const float *, const float *,
                                              long, float *, long, int *, int *, int, MpDevStatus *,
                                              cudaStream_t);
template cudaError_t launch_trsv_upper<double>(int, int, const double *, long, const double *,
                                               const double *, long, double *, long, int *, int *, int,
                                               MpDevStatus *, cudaStream_t);
