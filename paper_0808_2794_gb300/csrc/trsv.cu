// trsv.cu -- triangular solves with the low-precision factors,
// L y = P r and U z = y (Algorithm 1 steps 2-3 and 5-6; SGETRS, Section
// 3.1.1).
//
// GB300 design.  The factors are row-major.  Once per factorization the
// diagonal blocks of L and U are inverted at a large block size BI (1024
// rows in FP32 for n >= 2048): 128-row (64 in FP64) blocks are inverted by
// substitution, then neighbours are merged level by level with batched
// GEMMs (X21 = -X22 L21 X11 for L, X12 = -X11 U12 X22 for U).  A solve is
// then n/BI dependent steps, each y_b = inv(D_b) acc_b (a BI x BI product)
// followed by acc_r -= W[r, block b] y_b for the rows still to be solved.
// One persistent cooperative kernel runs them as a dataflow: a small group of
// CTAs follows the chain (the product with the inverse, then the next block's
// rows), the rest stream the remaining block columns from a work queue, and
// counters with bounded waits (MP_FLAG_TIMEOUT instead of a hang) order them.
//
// The right-hand side r (FP64) is scaled by s = 2^ceil(log2 ||r||inf) before
// it is rounded to the working precision (exact power-of-two scaling keeps
// tiny late residuals out of the subnormal range).
#include "common.cuh"
#include "kernels.cuh"

namespace {

constexpr int kMaxRhs = 8;
constexpr int kThreads = 256;

__device__ __forceinline__ double pow2_ceil(double v) {
    if (!(v > 0.0) || !(v <= 1.79769313486231570815e308)) return 1.0;
    int e;
    const double m = frexp(v, &e);
    return (m == 0.5) ? ldexp(1.0, e - 1) : ldexp(1.0, e);
}

template <typename T> constexpr int base_bs() { return sizeof(T) == 4 ? 128 : 64; }

// ---- inverses of the base diagonal blocks, written into the BI x BI layout
template <typename T, int BS>
__global__ void __launch_bounds__(BS)
base_inverse_kernel(int n, int BI, const T *__restrict__ W, long ldw, T *__restrict__ Linv, T *__restrict__ Uinv,
                    int lower_unit, int upper_unit) {
    extern __shared__ __align__(16) unsigned char raw[];
    T(*blk)[BS + 1] = reinterpret_cast<T(*)[BS + 1]>(raw);
    T(*x)[BS + 1] = reinterpret_cast<T(*)[BS + 1]>(raw + sizeof(T) * BS * (BS + 1));
    const int g = blockIdx.x, c = threadIdx.x;
    const int r0 = g * BS;
    const int bs = min(BS, n - r0);
    const int big = r0 / BI, o = r0 - big * BI;
    const long dst = (long)big * BI * BI + (long)o * BI + o;  // top-left of the sub-block
    for (int i = 0; i < BS; ++i) {
        const bool in = (i < bs) && (c < bs);
        blk[i][c] = in ? W[(long)(r0 + i) * ldw + r0 + c] : T(i == c ? 1 : 0);
    }
    __syncthreads();
    // lower: x_i = (delta_ic - sum_{l<i} L_il x_l) / L_ii, L_ii = 1 when unit
    // (thread c owns column c)
    for (int i = 0; i < BS; ++i) {
        T s = T(i == c ? 1 : 0);
        for (int l = c; l < i; ++l) s = fma(-blk[i][l], x[l][c], s);
        x[i][c] = (i < c) ? T(0) : (lower_unit ? s : s / blk[i][i]);
    }
    for (int i = 0; i < bs; ++i)
        if (c < bs) Linv[dst + (long)i * BI + c] = x[i][c];
    // upper: x_i = (delta_ic - sum_{l>i} U_il x_l) / U_ii, U_ii = 1 when unit
    for (int i = BS - 1; i >= 0; --i) {
        T s = T(i == c ? 1 : 0);
        for (int l = i + 1; l <= c; ++l) s = fma(-blk[i][l], x[l][c], s);
        x[i][c] = (i > c) ? T(0) : (upper_unit ? s : s / blk[i][i]);
    }
    for (int i = 0; i < bs; ++i)
        if (c < bs) Uinv[dst + (long)i * BI + c] = x[i][c];
}

// Vector type of 16 bytes.
template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; };
template <> struct Vec16<double> { using type = double2; };

// Dot products of one row segment (bs <= 1024 elements for FP32, <= 512 for
// FP64, 16-byte aligned) with nrhs vectors staged in shared memory (stride BI,
// zero beyond bs).  Each lane issues all its 16-byte loads before any FMA, so a
// row costs one memory latency.  Returns the warp-reduced sums in every lane.
template <typename T, bool STREAM, int NR>
__device__ __forceinline__ void row_dot(const T *__restrict__ src, int bs, const T *vs, int BI, int nrhs,
                                        T (&sum)[NR]) {
    using V = typename Vec16<T>::type;
    constexpr int VW = 16 / sizeof(T);
    constexpr int STRIDE = 32 * VW;
    constexpr int NQ = (sizeof(T) == 4 ? 1024 : 512) / STRIDE;
    const int lane = threadIdx.x & 31;
    T w[NQ][VW];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const int k = q * STRIDE + lane * VW;
        if (k + VW <= bs) {
            const V v = STREAM ? __ldcs(reinterpret_cast<const V *>(src + k)) : *reinterpret_cast<const V *>(src + k);
            const T *e = reinterpret_cast<const T *>(&v);
#pragma unroll
            for (int t = 0; t < VW; ++t) w[q][t] = e[t];
        } else {
#pragma unroll
            for (int t = 0; t < VW; ++t) w[q][t] = (k + t < bs) ? src[k + t] : T(0);
        }
    }
#pragma unroll
    for (int h = 0; h < NR; ++h) {
        T acc = T(0);
        if (h < nrhs) {
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const int k = q * STRIDE + lane * VW;
                if (k < bs) {
                    const V y = *reinterpret_cast<const V *>(vs + h * BI + k);
                    const T *ye = reinterpret_cast<const T *>(&y);
#pragma unroll
                    for (int t = 0; t < VW; ++t) acc = fma(w[q][t], ye[t], acc);
                }
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        }
        sum[h] = acc;
    }
}

// ---- the dataflow solve ----------------------------------------------------
// Blocks of BI rows are solved in order (first to last for L, last to first
// for U); a block's rows are split into chunks of RC rows.  Work items:
//   A(s)       y_b = inv(D_b) acc_b for block b = block(s), chunk by chunk
//   near(s)    acc_c -= W[c rows, block b] y_b for c = block(s + 1)
//   far(s, t)  the same for c = block(t), t >= s + 2
// A small group of "critical" CTAs runs A and near for every step in turn
// (the dependency chain); the other CTAs take the far items from a queue in
// the order (s, t, chunk) and stream the bulk of the factor meanwhile.  Each
// chunk's updates are applied in step order (a per-chunk counter), so every
// row sees the same sequence of subtractions as a step-by-step solve and the
// result does not depend on the schedule.  Counters (device memory, zeroed
// before the launch):
//   ycnt[b]   chunks of y_b written        updcnt[b]  chunk updates applied to block b
//   chunk[b][j] updates applied to chunk j of block b (release/acquire)
// Waits are bounded: after about a second a CTA records MP_FLAG_TIMEOUT,
// raises the abort word and returns; every wait also gives up on abort.
constexpr int kRC = 8;   // rows per chunk: the chain's items are 8 rows x BI of the factor (32 KB in FP32)
constexpr int kFG = 2;   // chunks per streaming item (16 rows)

struct TrsvSync {
    unsigned bar_count, bar_gen, qhead, abort, ncrit, pad[3];
    // followed by ycnt[nbi], updcnt[nbi], chunk[nbi * CH] (unsigned)
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Thread 0 waits until *p >= target (bounded); the CTA learns the outcome.
__device__ __forceinline__ bool wait_geq(const unsigned *p, unsigned target, TrsvSync *sy, MpDevStatus *st,
                                         bool *abort_s) {
    if (threadIdx.x == 0) {
        if (ld_acquire(p) < target) {
            const unsigned long long t0 = global_ns();
            long long polls = 0;
            while (ld_acquire(p) < target) {
                if (ld_acquire(&sy->abort) || ++polls > (1LL << 24) || global_ns() - t0 > 1000000000ULL) {
                    if (!ld_acquire(&sy->abort)) {
                        mp_flag(st, MP_FLAG_TIMEOUT);
                        atomicExch(&st->timeout_site, 2);
                        atomicExch(&sy->abort, 1u);
                    }
                    *abort_s = true;
                    break;
                }
                __nanosleep(64);
            }
        }
    }
    __syncthreads();
    return !*abort_s;
}

// acc[rows] -= F[rows, block] v for the rows [ra, rb) (a warp per row).
template <typename T, int NR>
__device__ __forceinline__ void update_rows(const T *F, long ldf, int coff, int bs, const T *vs, int BI, int nrhs,
                                            int ra, int rb, T *acc, int n, bool stream) {
    const int lane = threadIdx.x & 31;
    for (int r = ra + (threadIdx.x >> 5); r < rb; r += kThreads / 32) {
        T sum[NR];
        if (stream)
            row_dot<T, true, NR>(F + (long)r * ldf + coff, bs, vs, BI, nrhs, sum);
        else
            row_dot<T, false, NR>(F + (long)r * ldf + coff, bs, vs, BI, nrhs, sum);
        if (lane == 0)
#pragma unroll
            for (int h = 0; h < NR; ++h)
                if (h < nrhs) acc[(long)h * n + r] -= sum[h];
    }
}

// nrhs vectors of the block [r0, r0 + bs) into shared memory (stride BI,
// zero beyond bs), past L1: other CTAs wrote them in this launch.
template <typename T>
__device__ __forceinline__ void stage_vec(const T *src, long ld, int r0, int bs, int BI, int nrhs, T *vs) {
    for (int idx = threadIdx.x; idx < nrhs * BI; idx += kThreads) {
        const int h = idx / BI, k = idx - h * BI;
        vs[idx] = k < bs ? __ldcg(src + (long)h * ld + r0 + k) : T(0);
    }
    __syncthreads();
}

template <typename T, bool LOWER, int NR>
__global__ void __launch_bounds__(kThreads, NR <= 2 ? 4 : 2)
trsv_dataflow_kernel(int n, int nrhs, int BI, const T *__restrict__ W, long ldw, const T *__restrict__ Inv,
                     const double *__restrict__ R, long ldr, const int *__restrict__ perm,
                     const double *__restrict__ rnorm, const T *__restrict__ Yin, long ldyin,
                     T *__restrict__ Yout, long ldyout, T *__restrict__ acc, unsigned *sync, int crit_sms,
                     MpDevStatus *st) {
    extern __shared__ __align__(16) unsigned char raw[];
    T *vs = reinterpret_cast<T *>(raw);  // nrhs x BI vector of the current block
    __shared__ bool abort_s;
    __shared__ unsigned item_s, crit_s;
    TrsvSync *sy = reinterpret_cast<TrsvSync *>(sync);
    const int nbi = (n + BI - 1) / BI, CH = BI / kRC;
    unsigned *ycnt = sync + 8, *updcnt = ycnt + nbi, *chunk = updcnt + nbi;
    // the chain's group: the CTAs resident on the first crit_sms SMs, so
    // that no streaming CTA competes with them for an SM's load bandwidth
    if (threadIdx.x == 0) {
        abort_s = false;
        unsigned smid;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
        crit_s = (int)smid < crit_sms ? atomicAdd(&sy->ncrit, 1u) : 0xFFFFFFFFu;
    }
    const long gtid = (long)blockIdx.x * kThreads + threadIdx.x;
    const long gthreads = (long)gridDim.x * kThreads;
    auto block_of = [&](int s) { return LOWER ? s : nbi - 1 - s; };

    // acc = right-hand side (P r / s for L; y for U)
    for (long idx = gtid; idx < (long)nrhs * n; idx += gthreads) {
        const int h = (int)(idx / n), r = (int)(idx - (long)h * n);
        T v;
        if (LOWER) {
            const double s = pow2_ceil(rnorm[h]);
            v = (T)(R[(long)h * ldr + (perm ? perm[r] : r)] / s);
        } else {
            v = Yin[(long)h * ldyin + r];
        }
        acc[(long)h * n + r] = v;
    }
    if (!grid_barrier(&sy->bar_count, &sy->bar_gen, st, &abort_s)) return;
    int ncrit = (int)ld_acquire(&sy->ncrit);
    int ci = (int)crit_s;
    if (ncrit == 0 || ncrit >= (int)gridDim.x) {  // placement left no split: decide by index
        ncrit = max(1, min(CH, (int)gridDim.x / 4));
        ci = (int)blockIdx.x < ncrit ? (int)blockIdx.x : -1;
    }
    if (ci >= 0 && ci < ncrit) {
        // ---- the chain: A(s), then near(s), for every step
        for (int s = 0; s < nbi; ++s) {
            const int b = block_of(s), r0 = b * BI, bs = min(BI, n - r0);
            const T *D = Inv + (long)b * BI * BI;
            if (!wait_geq(&updcnt[b], (unsigned)(s * CH), sy, st, &abort_s)) return;
            stage_vec<T>(acc, n, r0, bs, BI, nrhs, vs);
            unsigned mine = 0;
            for (int j = ci; j < CH; j += ncrit) {
                const int ra = min(bs, j * kRC), rb = min(bs, ra + kRC);
                const int lane = threadIdx.x & 31;
                for (int r = ra + (threadIdx.x >> 5); r < rb; r += kThreads / 32) {
                    T sum[NR];
                    row_dot<T, false, NR>(D + (long)r * BI, bs, vs, BI, nrhs, sum);
                    if (lane == 0)
#pragma unroll
                        for (int h = 0; h < NR; ++h)
                            if (h < nrhs) Yout[(long)h * ldyout + r0 + r] = sum[h];
                }
                ++mine;
            }
            __syncthreads();
            if (threadIdx.x == 0 && mine) {
                __threadfence();
                atomicAdd(&ycnt[b], mine);
            }
            if (s + 1 == nbi) break;
            // near(s): the next block's rows
            const int c = block_of(s + 1), c0 = c * BI, cs = min(BI, n - c0);
            if (!wait_geq(&ycnt[b], (unsigned)CH, sy, st, &abort_s)) return;
            stage_vec<T>(Yout, ldyout, r0, bs, BI, nrhs, vs);
            for (int j = ci; j < CH; j += ncrit) {
                if (!wait_geq(&chunk[c * CH + j], (unsigned)s, sy, st, &abort_s)) return;
                const int ra = min(cs, j * kRC), rb = min(cs, ra + kRC);
                update_rows<T, NR>(W, ldw, r0, bs, vs, BI, nrhs, c0 + ra, c0 + rb, acc, n, true);
                __syncthreads();
                if (threadIdx.x == 0) {
                    __threadfence();
                    st_release(&chunk[c * CH + j], (unsigned)(s + 1));
                    atomicAdd(&updcnt[c], 1u);
                }
            }
        }
        return;
    }
    // ---- the far updates: items (s, t, j), t >= s + 2, taken in order
    const int NG = (CH + kFG - 1) / kFG;  // streaming items per block
    const long nfar = nbi >= 3 ? (long)(nbi - 2) * (nbi - 1) / 2 * NG : 0;
    int staged = -1;
    // the next item is claimed while the current one is processed
    if (threadIdx.x == 0) item_s = atomicAdd(&sy->qhead, 1u);
    __syncthreads();
    long q = item_s;
    __syncthreads();
    for (;;) {
        if (q >= nfar) break;
        unsigned next = 0;
        if (threadIdx.x == 0) next = atomicAdd(&sy->qhead, 1u);
        // decode: step s has (nbi - s - 2) * NG items
        long rem = q;
        int s = 0;
        while (rem >= (long)(nbi - s - 2) * NG) {
            rem -= (long)(nbi - s - 2) * NG;
            ++s;
        }
        const int t = s + 2 + (int)(rem / NG), j0 = (int)(rem % NG) * kFG, j1 = min(CH, j0 + kFG);
        const int b = block_of(s), r0 = b * BI, bs = min(BI, n - r0);
        const int c = block_of(t), c0 = c * BI, cs = min(BI, n - c0);
        if (staged != s) {
            if (!wait_geq(&ycnt[b], (unsigned)CH, sy, st, &abort_s)) return;
            stage_vec<T>(Yout, ldyout, r0, bs, BI, nrhs, vs);
            staged = s;
        }
        for (int j = j0; j < j1; ++j)
            if (!wait_geq(&chunk[c * CH + j], (unsigned)s, sy, st, &abort_s)) return;
        const int ra = min(cs, j0 * kRC), rb = min(cs, j1 * kRC);
        update_rows<T, NR>(W, ldw, r0, bs, vs, BI, nrhs, c0 + ra, c0 + rb, acc, n, true);
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            for (int j = j0; j < j1; ++j) st_release(&chunk[c * CH + j], (unsigned)(s + 1));
            atomicAdd(&updcnt[c], (unsigned)(j1 - j0));
            item_s = next;
        }
        __syncthreads();
        q = item_s;
        __syncthreads();
    }
}

int num_sms_cached() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 148;
    }
    return sms;
}

template <typename T, bool LOWER>
cudaError_t launch_persistent(int n, int nrhs, int BI, const T *W, long ldw, const T *Inv, const double *R, long ldr,
                              const int *perm, const double *rnorm, const T *Yin, long ldyin, T *Yout, long ldyout,
                              T *acc, unsigned *sync, MpDevStatus *st, cudaStream_t s) {
    if (n <= 0 || nrhs <= 0) return cudaSuccess;
    if (nrhs > kMaxRhs) return cudaErrorInvalidValue;
    // the right-hand-side count padded to 1, 2, 4 or 8 (fewer registers, so
    // more rows in flight per SM)
    auto kern = nrhs <= 1 ? trsv_dataflow_kernel<T, LOWER, 1>
                          : nrhs <= 2 ? trsv_dataflow_kernel<T, LOWER, 2>
                                      : nrhs <= 4 ? trsv_dataflow_kernel<T, LOWER, 4>
                                                  : trsv_dataflow_kernel<T, LOWER, 8>;
    const int nr = nrhs <= 1 ? 1 : nrhs <= 2 ? 2 : nrhs <= 4 ? 4 : 8;
    const size_t smem = sizeof(T) * (size_t)nr * BI;  // the vector of the current block
    cudaError_t e = mp_smem_attr(kern, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int grid = num_sms_cached() * std::min(per_sm, 4);
    // the chain's group: the CTAs on a quarter of the SMs
    int crit_sms = std::max(1, num_sms_cached() / 4);
    if (grid < 2) return cudaErrorInvalidConfiguration;
    e = cudaMemsetAsync(sync, 0, trsv_sync_bytes<T>(n), s);
    if (e != cudaSuccess) return e;
    void *args[] = {(void *)&n,    (void *)&nrhs,  (void *)&BI,    (void *)&W,      (void *)&ldw,
                    (void *)&Inv,  (void *)&R,     (void *)&ldr,   (void *)&perm,   (void *)&rnorm,
                    (void *)&Yin,  (void *)&ldyin, (void *)&Yout,  (void *)&ldyout, (void *)&acc,
                    (void *)&sync, (void *)&crit_sms, (void *)&st};
    mp_note_launch();
    return cudaLaunchCooperativeKernel((const void *)kern, dim3(grid), dim3(kThreads), args, smem, s);
}

// Timeout path of the grid barrier, for the self-test: every CTA arrives,
// but a generation needs one arrival more than the grid has, so no CTA can
// pass; each gives up after limit_ns and records the timeout (site 2).
__global__ void selftest_grid_barrier_kernel(unsigned *count, unsigned *gen, MpDevStatus *st,
                                             unsigned long long limit_ns, int *passed) {
    __shared__ bool abort_s;
    if (threadIdx.x == 0) abort_s = false;
    __syncthreads();
    if (grid_barrier(count, gen, st, &abort_s, limit_ns, gridDim.x + 1) && threadIdx.x == 0) atomicAdd(passed, 1);
}

}  // namespace

cudaError_t launch_selftest_grid_barrier(unsigned *bar, MpDevStatus *st, unsigned long long limit_ns, int *passed,
                                         cudaStream_t s) {
    unsigned *count = bar, *gen = bar + 1;
    void *args[] = {&count, &gen, &st, &limit_ns, &passed};
    mp_note_launch();
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(selftest_grid_barrier_kernel), dim3(2), dim3(32),
                                       args, 0, s);
}

template <typename T>
int trsv_inverse_block(int n) {
    const int base = base_bs<T>();
    const int top = sizeof(T) == 4 ? 1024 : 512;
    int bi = base;
    while (bi < top && bi < n) bi *= 2;
    return bi;
}
template int trsv_inverse_block<float>(int);
template int trsv_inverse_block<double>(int);

template <typename T>
size_t trsv_inverse_bytes(int n) {
    const int BI = trsv_inverse_block<T>(n);
    const size_t nbi = (size_t)(n + BI - 1) / BI;
    return nbi * BI * BI * sizeof(T);
}
template size_t trsv_inverse_bytes<float>(int);
template size_t trsv_inverse_bytes<double>(int);

template <typename T>
size_t trsv_sync_bytes(int n) {
    const int BI = trsv_inverse_block<T>(n);
    const size_t nbi = (size_t)(std::max(n, 1) + BI - 1) / BI;
    return sizeof(unsigned) * (8 + 2 * nbi + nbi * (size_t)(BI / kRC));
}
template size_t trsv_sync_bytes<float>(int);
template size_t trsv_sync_bytes<double>(int);

template <typename T>
size_t trsv_tmp_bytes(int n) {
    const int BI = trsv_inverse_block<T>(n);
    const size_t nbi = (size_t)(n + BI - 1) / BI;
    return nbi * (size_t)BI * BI / 4 * sizeof(T) + 256;
}
template size_t trsv_tmp_bytes<float>(int);
template size_t trsv_tmp_bytes<double>(int);

// Builds inv(L_bb) and inv(U_bb) for the BI x BI diagonal blocks of the
// row-major factors in W.  tmp holds trsv_tmp_bytes<T>(n).
template <typename T>
cudaError_t launch_build_inverses(int n, const T *W, long ldw, T *Linv, T *Uinv, T *tmp, cudaStream_t s,
                                  bool lower_unit, bool upper_unit) {
    if (n <= 0) return cudaSuccess;
    constexpr int BS = base_bs<T>();
    const int BI = trsv_inverse_block<T>(n);
    const int nbi = (n + BI - 1) / BI;
    const size_t bytes = (size_t)nbi * BI * BI * sizeof(T);
    cudaError_t e = cudaMemsetAsync(Linv, 0, bytes, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(Uinv, 0, bytes, s);
    if (e != cudaSuccess) return e;
    {
        auto kern = base_inverse_kernel<T, BS>;
        const size_t smem = 2 * sizeof(T) * BS * (BS + 1);
        e = mp_smem_attr(kern, smem);
        if (e != cudaSuccess) return e;
        mp_note_launch();
        kern<<<(n + BS - 1) / BS, BS, smem, s>>>(n, BI, W, ldw, Linv, Uinv, lower_unit ? 1 : 0, upper_unit ? 1 : 0);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const int nfull = n / BI;
    const long BB = (long)BI * BI;
    for (int h = BS; h < BI; h *= 2) {
        const int pairs = BI / (2 * h);
        // full BI blocks: batched over (block, pair)
        if (nfull > 0) {
            const int batch = nfull * pairs;
            const long wo = (long)BI * ldw + BI, wi = (long)2 * h * ldw + 2 * h;   // W strides
            const long io = BB, ii = (long)2 * h * BI + 2 * h;                      // inverse strides
            const long to = (long)pairs * h * h, ti = (long)h * h;                  // tmp strides
            // L: T = L21 X11 ; X21 = -X22 T
            e = launch_gemm_batched<T>(h, h, h, T(1), T(0), W + (long)h * ldw, ldw, Linv, BI, tmp, h, batch, pairs,
                                       wo, wi, io, ii, to, ti, s);
            if (e != cudaSuccess) return e;
            e = launch_gemm_batched<T>(h, h, h, T(-1), T(0), Linv + (long)h * BI + h, BI, tmp, h,
                                       Linv + (long)h * BI, BI, batch, pairs, io, ii, to, ti, io, ii, s);
            if (e != cudaSuccess) return e;
            // U: T = U12 X22 ; X12 = -X11 T
            e = launch_gemm_batched<T>(h, h, h, T(1), T(0), W + h, ldw, Uinv + (long)h * BI + h, BI, tmp, h, batch,
                                       pairs, wo, wi, io, ii, to, ti, s);
            if (e != cudaSuccess) return e;
            e = launch_gemm_batched<T>(h, h, h, T(-1), T(0), Uinv, BI, tmp, h, Uinv + h, BI, batch, pairs, io, ii,
                                       to, ti, io, ii, s);
            if (e != cudaSuccess) return e;
        }
        // the partial last block: pair by pair with clipped sizes
        if (nfull < nbi) {
            const int base = nfull * BI;
            T *Lb = Linv + (long)nfull * BB, *Ub = Uinv + (long)nfull * BB;
            for (int p = 0; p < pairs; ++p) {
                const int o1 = p * 2 * h, o2 = o1 + h;
                if (base + o2 >= n) break;
                const int h2 = std::min(h, n - (base + o2));
                const T *L21 = W + (long)(base + o2) * ldw + base + o1;
                const T *U12 = W + (long)(base + o1) * ldw + base + o2;
                e = launch_gemm_batched<T>(h2, h, h, T(1), T(0), L21, ldw, Lb + (long)o1 * BI + o1, BI, tmp, h, 1, 1,
                                           0, 0, 0, 0, 0, 0, s);
                if (e != cudaSuccess) return e;
                e = launch_gemm_batched<T>(h2, h, h2, T(-1), T(0), Lb + (long)o2 * BI + o2, BI, tmp, h,
                                           Lb + (long)o2 * BI + o1, BI, 1, 1, 0, 0, 0, 0, 0, 0, s);
                if (e != cudaSuccess) return e;
                e = launch_gemm_batched<T>(h, h2, h2, T(1), T(0), U12, ldw, Ub + (long)o2 * BI + o2, BI, tmp, h2, 1, 1,
                                           0, 0, 0, 0, 0, 0, s);
                if (e != cudaSuccess) return e;
                e = launch_gemm_batched<T>(h, h2, h, T(-1), T(0), Ub + (long)o1 * BI + o1, BI, tmp, h2,
                                           Ub + (long)o1 * BI + o2, BI, 1, 1, 0, 0, 0, 0, 0, 0, s);
                if (e != cudaSuccess) return e;
            }
        }
    }
    return cudaSuccess;
}
template cudaError_t launch_build_inverses<float>(int, const float *, long, float *, float *, float *, cudaStream_t,
                                                  bool, bool);
template cudaError_t launch_build_inverses<double>(int, const double *, long, double *, double *, double *,
                                                   cudaStream_t, bool, bool);

template <typename T>
cudaError_t launch_trsv_lower(int n, int nrhs, const T *W, long ldw, const T *Linv, const double *R, long ldr,
                              const int *perm, const double *rnorm, T *Y, long ldy, T *acc, unsigned *bar,
                              MpDevStatus *st, cudaStream_t s) {
    return launch_persistent<T, true>(n, nrhs, trsv_inverse_block<T>(n), W, ldw, Linv, R, ldr, perm, rnorm,
                                      nullptr, 0, Y, ldy, acc, bar, st, s);
}
template cudaError_t launch_trsv_lower<float>(int, int, const float *, long, const float *, const double *, long,
                                              const int *, const double *, float *, long, float *, unsigned *,
                                              MpDevStatus *, cudaStream_t);
template cudaError_t launch_trsv_lower<double>(int, int, const double *, long, const double *, const double *,
                                               long, const int *, const double *, double *, long, double *,
                                               unsigned *, MpDevStatus *, cudaStream_t);

template <typename T>
cudaError_t launch_trsv_upper(int n, int nrhs, const T *W, long ldw, const T *Uinv, const T *Y, long ldy, T *Z,
                              long ldz, T *acc, unsigned *bar, MpDevStatus *st, cudaStream_t s) {
    return launch_persistent<T, false>(n, nrhs, trsv_inverse_block<T>(n), W, ldw, Uinv, nullptr, 0, nullptr,
                                       nullptr, Y, ldy, Z, ldz, acc, bar, st, s);
}
template cudaError_t launch_trsv_upper<float>(int, int, const float *, long, const float *, const float *, long,
                                              float *, long, float *, unsigned *, MpDevStatus *, cudaStream_t);
template cudaError_t launch_trsv_upper<double>(int, int, const double *, long, const double *, const double *,
                                               long, double *, long, double *, unsigned *, MpDevStatus *,
                                               cudaStream_t);
