// trsv.cu -- triangular solves with the low-precision factors,
// L y = P r and U z = y (Algorithm 1 steps 2-3 and 5-6; SGETRS, Section
// 3.1.1).
//
// GB300 design.  The factors are row-major, so every block row of L (or U)
// is a set of contiguous row segments.  The n rows are cut into BS-row
// blocks (BS = 128 for FP32, 64 for FP64); the diagonal blocks are inverted
// once after the factorization, so that a block's own solve is a small
// parallel matrix-vector product.  The off-diagonal work of block row i is
// split into chunks of kChunk blocks; every (block row, chunk) pair is one
// CTA that streams its part of the row as soon as the blocks it needs are
// published (per-block flags), writes a partial sum to its own slot, and
// counts itself in.  The CTA that completes the last chunk of a row adds the
// slots in a fixed order (deterministic), applies the inverted diagonal
// block and publishes the block.  CTAs take work items from an atomic ticket
// in dependency order, so a CTA only waits on items that already run; every
// wait is bounded and reports MP_FLAG_TIMEOUT if it gives up.
//
// The right-hand side r (FP64) is scaled by s = 2^ceil(log2 ||r||inf) before
// it is rounded to the working precision (exact power-of-two scaling keeps
// tiny late residuals out of the subnormal range).
#include "common.cuh"
#include "kernels.cuh"

namespace {

constexpr int kMaxRhs = 8;
constexpr int kChunk = 8;  // dependency blocks per CTA

__device__ __forceinline__ double pow2_ceil(double v) {
    if (!(v > 0.0) || !(v <= 1.79769313486231570815e308)) return 1.0;
    int e;
    const double m = frexp(v, &e);
    return (m == 0.5) ? ldexp(1.0, e - 1) : ldexp(1.0, e);
}

// ---- inverses of the diagonal blocks ---------------------------------------
template <typename T, int BS>
__global__ void __launch_bounds__(BS)
diag_inverse_kernel(int n, const T *__restrict__ W, long ldw, T *__restrict__ Linv, T *__restrict__ Uinv) {
    extern __shared__ __align__(16) unsigned char raw[];
    T(*blk)[BS + 1] = reinterpret_cast<T(*)[BS + 1]>(raw);
    T(*x)[BS + 1] = reinterpret_cast<T(*)[BS + 1]>(raw + sizeof(T) * BS * (BS + 1));
    const int b = blockIdx.x, c = threadIdx.x;
    const int r0 = b * BS;
    const int bs = min(BS, n - r0);
    for (int i = 0; i < BS; ++i) {
        const bool in = (i < bs) && (c < bs);
        blk[i][c] = in ? W[(long)(r0 + i) * ldw + r0 + c] : T(i == c ? 1 : 0);
    }
    __syncthreads();
    // unit lower: x_i = delta_ic - sum_{l<i} L_il x_l (thread c owns column c)
    for (int i = 0; i < BS; ++i) {
        T s = T(i == c ? 1 : 0);
        for (int l = c; l < i; ++l) s = fma(-blk[i][l], x[l][c], s);
        x[i][c] = (i < c) ? T(0) : s;
    }
    T *Lo = Linv + (long)b * BS * BS;
    for (int i = 0; i < BS; ++i) Lo[i * BS + c] = x[i][c];
    // upper: x_i = (delta_ic - sum_{l>i} U_il x_l) / U_ii
    for (int i = BS - 1; i >= 0; --i) {
        T s = T(i == c ? 1 : 0);
        for (int l = i + 1; l <= c; ++l) s = fma(-blk[i][l], x[l][c], s);
        x[i][c] = (i > c) ? T(0) : s / blk[i][i];
    }
    T *Uo = Uinv + (long)b * BS * BS;
    for (int i = 0; i < BS; ++i) Uo[i * BS + c] = x[i][c];
}

__host__ __device__ __forceinline__ int nchunks(int deps) { return (deps + kChunk - 1) / kChunk; }

// Work items of the block rows before solve position q (the row at position
// q has q dependencies): sum over q' < q of max(1, nchunks(q')).
__host__ __device__ __forceinline__ long items_before(int q) {
    if (q <= 0) return 0;
    const long C = kChunk;
    const long Q = q - 1;  // positions 1..Q contribute ceil(q'/C) each, position 0 one item
    const long full = Q / C, rem = Q % C;
    return 1 + C * full * (full + 1) / 2 + (full + 1) * rem;
}

// One CTA per (block row, chunk).  Thread (r = tid / TPR, part = tid % TPR)
// owns row r of the block and a BS/TPR-column segment of each block.
template <typename T, int BS, bool LOWER>
__global__ void __launch_bounds__(256)
trsv_chunk_kernel(int n, int nrhs, const T *__restrict__ W, long ldw, const T *__restrict__ Dinv,
                  const double *__restrict__ R, long ldr, const int *__restrict__ perm,
                  const double *__restrict__ rnorm, const T *__restrict__ Yin, long ldyin,
                  T *__restrict__ Yout, long ldyout, T *__restrict__ slots, int *flags, int *counts,
                  int *ticket, int epoch, long items_per_solve, MpDevStatus *st) {
    constexpr int TPR = 256 / BS;  // threads per row (2 for BS=128, 4 for BS=64)
    constexpr int SEG = BS / TPR;  // columns per thread per block
    __shared__ int s_q, s_c, s_ready;
    __shared__ bool s_ok, s_last;
    __shared__ T ys[kMaxRhs][BS];  // y of the current dependency block
    __shared__ T accs[kMaxRhs][BS];
    const int tid = threadIdx.x;
    const int r = tid / TPR, part = tid % TPR;
    const int nblk = (n + BS - 1) / BS;
    if (tid == 0) {
        const long t = (long)atomicAdd(ticket, 1) - (long)(epoch - 1) * items_per_solve;
        int lo = 0, hi = nblk - 1;  // largest q with items_before(q) <= t
        while (lo < hi) {
            const int mid = (lo + hi + 1) / 2;
            if (items_before(mid) <= t) lo = mid; else hi = mid - 1;
        }
        s_q = lo;
        s_c = (int)(t - items_before(lo));
        s_ok = true;
        s_last = false;
    }
    __syncthreads();
    const int q = s_q, c = s_c;
    const int i = LOWER ? q : nblk - 1 - q;  // block row
    const int row = i * BS + r;
    const bool rvalid = row < n;
    const int nch = nchunks(q);
    T part_acc[kMaxRhs];
#pragma unroll
    for (int h = 0; h < kMaxRhs; ++h) part_acc[h] = T(0);

    if (nch > 0) {
        // dependencies at solve positions [d0, d1); block column j = position
        // (lower) or nblk-1-position (upper)
        const int d0 = c * kChunk, d1 = min(q, d0 + kChunk);
        int ready = d0;
        for (int d = d0; d < d1; ++d) {
            const int j = LOWER ? d : nblk - 1 - d;
            if (d == ready) {
                if (tid == 0) {
                    const volatile int *vf = flags;
                    bool ok = wait_flag_geq(vf + j, epoch, st, 1);
                    int e = d + 1;
                    while (ok && e < d1 && vf[LOWER ? e : nblk - 1 - e] >= epoch) ++e;
                    __threadfence();
                    s_ready = e;
                    if (!ok) s_ok = false;
                }
                __syncthreads();
                if (!s_ok) break;
                ready = s_ready;
            }
            for (int idx = tid; idx < nrhs * BS; idx += 256) {  // stage y_j
                const int h = idx / BS, k = idx % BS;
                const int col = j * BS + k;
                ys[h][k] = col < n ? __ldcg(Yout + (long)h * ldyout + col) : T(0);
            }
            __syncthreads();
            if (rvalid) {
                const int c0 = j * BS + part * SEG;
                const T *wrow = W + (long)row * ldw + c0;
                T wv[SEG];
#pragma unroll
                for (int qq = 0; qq < SEG; ++qq) wv[qq] = (c0 + qq < n) ? wrow[qq] : T(0);
#pragma unroll
                for (int h = 0; h < kMaxRhs; ++h) {
                    if (h < nrhs) {
                        T acc = part_acc[h];
#pragma unroll
                        for (int qq = 0; qq < SEG; ++qq) acc = fma(wv[qq], ys[h][part * SEG + qq], acc);
                        part_acc[h] = acc;
                    }
                }
            }
            __syncthreads();  // ys is reused by the next block
        }
        if (!s_ok) return;  // timeout recorded in the status block
#pragma unroll
        for (int h = 0; h < kMaxRhs; ++h)
#pragma unroll
            for (int off = 1; off < TPR; off <<= 1) part_acc[h] += __shfl_xor_sync(0xffffffffu, part_acc[h], off);
        if (part == 0) {
            T *slot = slots + (items_before(q) + c) * kMaxRhs * BS;
            for (int h = 0; h < nrhs; ++h) slot[h * BS + r] = part_acc[h];
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) {
            const int old = atomicAdd(&counts[i], 1);
            s_last = (old + 1 == epoch * nch);
        }
        __syncthreads();
        if (!s_last) return;
        __threadfence();
    }
    // ---- the last chunk of block row i: acc = rhs - sum of the chunk partials
    if (part == 0) {
#pragma unroll 1
        for (int h = 0; h < nrhs; ++h) {
            T sum = T(0);
            for (int cc = 0; cc < nch; ++cc)
                sum += __ldcg(slots + ((items_before(q) + cc) * kMaxRhs + h) * BS + r);
            T rhs = T(0);
            if (rvalid) {
                if (LOWER) {
                    const double s = pow2_ceil(rnorm[h]);
                    rhs = (T)(R[(long)h * ldr + perm[row]] / s);
                } else {
                    rhs = Yin[(long)h * ldyin + row];
                }
            }
            accs[h][r] = rvalid ? rhs - sum : T(0);
        }
    }
    __syncthreads();
    // y_i = Dinv_i * acc
    const T *D = Dinv + (long)i * BS * BS + (long)r * BS + part * SEG;
    T dv[SEG];
#pragma unroll
    for (int qq = 0; qq < SEG; ++qq) dv[qq] = D[qq];
    for (int h = 0; h < nrhs; ++h) {
        T acc = T(0);
#pragma unroll
        for (int qq = 0; qq < SEG; ++qq) acc = fma(dv[qq], accs[h][part * SEG + qq], acc);
#pragma unroll
        for (int off = 1; off < TPR; off <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (part == 0 && rvalid) Yout[(long)h * ldyout + row] = acc;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) atomicExch(&flags[i], epoch);
}

}  // namespace

template <typename T>
int trsv_block_size() { return sizeof(T) == 4 ? 128 : 64; }
template int trsv_block_size<float>();
template int trsv_block_size<double>();

size_t trsv_slot_bytes(int n, int bs, size_t elem) {
    const int nblk = (n + bs - 1) / bs;
    return (size_t)items_before(nblk) * kMaxRhs * bs * elem;
}

template <typename T>
cudaError_t launch_diag_inverses(int n, const T *W, long ldw, T *Linv, T *Uinv, cudaStream_t s) {
    constexpr int BS = sizeof(T) == 4 ? 128 : 64;
    const int nblk = (n + BS - 1) / BS;
    if (nblk == 0) return cudaSuccess;
    auto kern = diag_inverse_kernel<T, BS>;
    const size_t smem = 2 * sizeof(T) * BS * (BS + 1);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    mp_note_launch();
    kern<<<nblk, BS, smem, s>>>(n, W, ldw, Linv, Uinv);
    return cudaGetLastError();
}
template cudaError_t launch_diag_inverses<float>(int, const float *, long, float *, float *, cudaStream_t);
template cudaError_t launch_diag_inverses<double>(int, const double *, long, double *, double *, cudaStream_t);

template <typename T>
cudaError_t launch_trsv_lower(int n, int nrhs, const T *W, long ldw, const T *Linv, const double *R, long ldr,
                              const int *perm, const double *rnorm, T *Y, long ldy, T *slots, int *flags,
                              int *counts, int *ticket, int epoch, MpDevStatus *st, cudaStream_t s) {
    constexpr int BS = sizeof(T) == 4 ? 128 : 64;
    if (nrhs > kMaxRhs) return cudaErrorInvalidValue;
    const int nblk = (n + BS - 1) / BS;
    if (nblk == 0) return cudaSuccess;
    const long items = items_before(nblk);
    mp_note_launch();
    trsv_chunk_kernel<T, BS, true><<<(unsigned)items, 256, 0, s>>>(n, nrhs, W, ldw, Linv, R, ldr, perm, rnorm,
                                                                   nullptr, 0, Y, ldy, slots, flags, counts,
                                                                   ticket, epoch, items, st);
    return cudaGetLastError();
}
template cudaError_t launch_trsv_lower<float>(int, int, const float *, long, const float *, const double *, long,
                                              const int *, const double *, float *, long, float *, int *, int *,
                                              int *, int, MpDevStatus *, cudaStream_t);
template cudaError_t launch_trsv_lower<double>(int, int, const double *, long, const double *, const double *,
                                               long, const int *, const double *, double *, long, double *, int *,
                                               int *, int *, int, MpDevStatus *, cudaStream_t);

template <typename T>
cudaError_t launch_trsv_upper(int n, int nrhs, const T *W, long ldw, const T *Uinv, const T *Y, long ldy, T *Z,
                              long ldz, T *slots, int *flags, int *counts, int *ticket, int epoch,
                              MpDevStatus *st, cudaStream_t s) {
    constexpr int BS = sizeof(T) == 4 ? 128 : 64;
    if (nrhs > kMaxRhs) return cudaErrorInvalidValue;
    const int nblk = (n + BS - 1) / BS;
    if (nblk == 0) return cudaSuccess;
    const long items = items_before(nblk);
    mp_note_launch();
    trsv_chunk_kernel<T, BS, false><<<(unsigned)items, 256, 0, s>>>(n, nrhs, W, ldw, Uinv, nullptr, 0, nullptr,
                                                                    nullptr, Y, ldy, Z, ldz, slots, flags, counts,
                                                                    ticket, epoch, items, st);
    return cudaGetLastError();
}
template cudaError_t launch_trsv_upper<float>(int, int, const float *, long, const float *, const float *, long,
                                              float *, long, float *, int *, int *, int *, int, MpDevStatus *,
                                              cudaStream_t);
template cudaError_t launch_trsv_upper<double>(int, int, const double *, long, const double *, const double *,
                                               long, double *, long, double *, int *, int *, int *, int,
                                               MpDevStatus *, cudaStream_t);
