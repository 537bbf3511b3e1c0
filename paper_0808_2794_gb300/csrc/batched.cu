// batched.cu -- many independent small systems (n <= 512) solved by one
// persistent launch: Algorithm 1 (Section 2.1) per system, with the
// factorization, the triangular solves, the FP64 residual and the update all
// inside one CTA.  Section 2.1 notes that for small problems the low-precision
// factorization stops paying off once the O(n^2) refinement costs about as
// much as the O(n^3) step; keeping every step of a system on one SM removes
// the per-step launch latency that makes small systems expensive.
//
// Systems are taken from a queue ordered by decreasing n^3 (longest first),
// one CTA per system at a time.  The working matrix W of a system is
// row-major FP32 (FP64 in the fallback pass), ld = round_up(n, 4), in global
// memory (L2-resident for these sizes); the current column panel and the
// U12 block of each outer step sit in shared memory.
//
//   convert     W = fl(A), ||A||inf (row sums in a fixed order), ||b||inf
//   panel       GEPP on rows k.., columns k..k+NB (argmax ties -> lowest row)
//   row moves   the panel's interchanges on the other columns of W
//   U12         L11^{-1} A12 (column per thread)
//   update      A22 -= fl_p(L21) fl_p(U12), FP32 products/accumulation
//   solves      y = L^{-1} P (r / s), z = U^{-1} y (32-row blocks)
//   residual    r = b - A x in FP64 (row per thread, fixed order)
//   test        the A1 rule of the single-system driver; stall -> fallback
//
// A system whose low-precision refinement fails is marked and re-solved by
// the same kernel instantiated for FP64 (Section 4's fallback).
#include "batched.cuh"
#include "batched_schedule.h"
#include "common.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

namespace {

constexpr int NT = 256;
constexpr int kMaxN = MP_BATCH_MAX_N;
constexpr int kMaxRhs = 8;

// 16-byte vector of T and its width
template <typename T> struct V16Of;
template <> struct V16Of<float> { using type = float4; };
template <> struct V16Of<double> { using type = double2; };
template <typename T> using V16 = typename V16Of<T>::type;
template <typename T> constexpr int VW16 = 16 / (int)sizeof(T);

template <typename T> struct BCfg;
template <> struct BCfg<float> { static constexpr int NB = 16; };
template <> struct BCfg<double> { static constexpr int NB = 16; };


__device__ __forceinline__ double pow2_ceil_d(double v) {
    if (!(v > 0.0) || !(v <= 1.79769313486231570815e308)) return 1.0;
    int e;
    const double m = frexp(v, &e);
    return (m == 0.5) ? ldexp(1.0, e - 1) : ldexp(1.0, e);
}

// Operand rounding of the trailing update (p = fp32: identity).
template <typename T>
__device__ __forceinline__ T round_p(T v, int prec) {
    if constexpr (sizeof(T) == 4) {
        if (prec == MP_PREC_BF16) return __bfloat162float(__float2bfloat16_rn(v));
        if (prec == MP_PREC_FP16) return __half2float(__float2half_rn(v));
    }
    return v;
}

struct Shared {
    double dred[NT / 32];
    int ired[NT / 32];
    double anorm;
    double bnorm[kMaxRhs], rnorm[kMaxRhs], xnorm[kMaxRhs], znorm[kMaxRhs], zprev[kMaxRhs];
    int piv, sys, stop, info;
    unsigned flags;
    int nmoves;
    int rowsrc[64], mdst[64], pv[64];  // composed row moves of one panel (<= 2 NB)
};

// Dynamic shared memory: panel, U12 block (also the solve vectors), x in
// FP64 for the residual, then the Shared block (8-byte aligned after the
// double array).
template <typename T>
constexpr size_t batched_smem_bytes() {
    constexpr int NB = BCfg<T>::NB;
    return sizeof(T) * (size_t)kMaxN * (NB + 1)       // panel
           + sizeof(T) * (size_t)NB * kMaxN           // U12 block / vectors
           + sizeof(double) * (size_t)kMaxN * kMaxRhs // x (FP64) for the residual
           + sizeof(Shared);                          // reductions, scalars, row moves
}
static_assert((sizeof(float) * (size_t)kMaxN * 17 + sizeof(float) * 16 * kMaxN) % 8 == 0, "alignment");
static_assert((sizeof(double) * (size_t)kMaxN * 17 + sizeof(double) * 16 * kMaxN) % 8 == 0, "alignment");

// Block-wide max of a non-negative double (NaN counts as +inf).
__device__ double block_max(double v, Shared &sh) {
    if (v != v) v = __longlong_as_double(0x7ff0000000000000LL);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh.dred[threadIdx.x >> 5] = v;
    __syncthreads();
    double m = 0.0;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) m = fmax(m, sh.dred[w]);
    return m;
}

template <typename T, int NB>
__device__ void lu_factor(const BatchSys &d, T *W, int ldw, T *P, T *Us, Shared &sh, int prec) {
    const int n = d.n, tid = threadIdx.x;
    for (int k = 0; k < n; k += NB) {
        const int nb = min(NB, n - k), m = n - k;
        // panel rows k.. x columns k..k+nb into shared memory
        for (int e = tid; e < m * nb; e += NT) {
            const int r = e / nb, c = e - r * nb;
            P[r * (NB + 1) + c] = W[(long)(k + r) * ldw + k + c];
        }
        __syncthreads();
        for (int j = 0; j < nb; ++j) {
            // argmax |P[r][j]| over r >= j, ties to the smallest r, NaN as +inf
            double best = -1.0;
            int bi = m;
            for (int r = j + tid; r < m; r += NT) {
                double a = fabs((double)P[r * (NB + 1) + j]);
                if (a != a) a = __longlong_as_double(0x7ff0000000000000LL);
                if (a > best) { best = a; bi = r; }
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const double ob = __shfl_xor_sync(0xffffffffu, best, off);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            if ((tid & 31) == 0) { sh.dred[tid >> 5] = best; sh.ired[tid >> 5] = bi; }
            __syncthreads();
            if (tid == 0) {
                double b = sh.dred[0];
                int i = sh.ired[0];
                for (int w = 1; w < NT / 32; ++w)
                    if (sh.dred[w] > b || (sh.dred[w] == b && sh.ired[w] < i)) { b = sh.dred[w]; i = sh.ired[w]; }
                sh.piv = i;
                d.ipiv[k + j] = k + i + 1;
                const T pv = P[i * (NB + 1) + j];
                if (!(pv != T(0)) || !(fabs((double)pv) <= 1.79769313486231570815e308)) {
                    sh.flags |= MP_FLAG_LOWP_BREAKDOWN;
                    if (sh.info == 0) sh.info = k + j + 1;
                }
            }
            __syncthreads();
            const int p = sh.piv;
            if (p != j && tid < nb) {
                const T t = P[j * (NB + 1) + tid];
                P[j * (NB + 1) + tid] = P[p * (NB + 1) + tid];
                P[p * (NB + 1) + tid] = t;
            }
            __syncthreads();
            const T dg = P[j * (NB + 1) + j];
            const bool ok = dg != T(0) && fabs((double)dg) <= 1.79769313486231570815e308;
            if (ok)
                for (int r = j + 1 + tid; r < m; r += NT) P[r * (NB + 1) + j] = P[r * (NB + 1) + j] / dg;
            __syncthreads();
            if (ok)
                for (int r = j + 1 + tid; r < m; r += NT) {
                    T *pr = P + r * (NB + 1);
                    const T lr = pr[j];
                    for (int c = j + 1; c < nb; ++c) pr[c] = fma(-lr, P[j * (NB + 1) + c], pr[c]);
                }
            __syncthreads();
        }
        for (int e = tid; e < m * nb; e += NT) {
            const int r = e / nb, c = e - r * nb;
            W[(long)(k + r) * ldw + k + c] = P[r * (NB + 1) + c];
        }
        // the panel's interchanges on the columns outside it: composed into at
        // most 2 nb (destination, source) row moves, then every thread moves
        // whole columns with all loads in flight before the stores
        if (tid == 0) {
            int *src = sh.rowsrc;  // rows k.. : which original row is now there
            int nmv = 0;
            for (int j = 0; j < nb; ++j) {
                const int p = d.ipiv[k + j] - 1 - k;
                // rows are looked up by position; untouched rows hold themselves
                int a = -1, b = -1;
                for (int t = 0; t < nmv; ++t) {
                    if (sh.mdst[t] == j) a = t;
                    if (sh.mdst[t] == p) b = t;
                }
                if (p == j) continue;
                if (a < 0) { sh.mdst[nmv] = j; src[nmv] = j; a = nmv++; }
                if (b < 0) { sh.mdst[nmv] = p; src[nmv] = p; b = nmv++; }
                const int t = src[a];
                src[a] = src[b];
                src[b] = t;
            }
            sh.nmoves = nmv;
        }
        __syncthreads();
        const int nmv = sh.nmoves;
        for (int c = tid; c < n; c += NT) {
            if (c >= k && c < k + nb) continue;
            T v[2 * NB];
#pragma unroll
            for (int t = 0; t < 2 * NB; ++t)
                if (t < nmv) v[t] = W[(long)(k + sh.rowsrc[t]) * ldw + c];
#pragma unroll
            for (int t = 0; t < 2 * NB; ++t)
                if (t < nmv) W[(long)(k + sh.mdst[t]) * ldw + c] = v[t];
        }
        if (tid < nmv) sh.pv[tid] = d.perm[k + sh.rowsrc[tid]];
        __syncthreads();
        if (tid < nmv) d.perm[k + sh.mdst[tid]] = sh.pv[tid];
        __syncthreads();
        const int rest = n - k - nb;
        if (rest <= 0) continue;
        // U12 = L11^{-1} A12 (unit lower L11 from the panel), one column per thread
        for (int c = tid; c < rest; c += NT) {
            T u[NB];
#pragma unroll
            for (int i = 0; i < NB; ++i) u[i] = i < nb ? W[(long)(k + i) * ldw + k + nb + c] : T(0);
#pragma unroll
            for (int i = 1; i < NB; ++i)
#pragma unroll
                for (int l = 0; l < i; ++l) u[i] = fma(-P[i * (NB + 1) + l], u[l], u[i]);
#pragma unroll
            for (int i = 0; i < NB; ++i)
                if (i < nb) {
                    W[(long)(k + i) * ldw + k + nb + c] = u[i];
                    Us[i * kMaxN + c] = round_p(u[i], prec);
                }
        }
        // L21 rounded to p in place (the stored factor keeps FP32: the
        // rounded copy lives only in the panel buffer)
        if (prec != MP_PREC_FP32)
            for (int e = tid; e < rest * nb; e += NT) {
                const int r = nb + e / nb, c = e % nb;
                P[r * (NB + 1) + c] = round_p(P[r * (NB + 1) + c], prec);
            }
        __syncthreads();
        // A22 -= L21 U12: 4 x 4 outputs per thread, 64 x 64 tiles
        const int ty = tid >> 4, tx = tid & 15;
        for (int r0 = 0; r0 < rest; r0 += 64)
            for (int c0 = 0; c0 < rest; c0 += 64) {
                T acc[4][4];
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const int r = r0 + ty * 4 + a;
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const int c = c0 + tx * 4 + b;
                        acc[a][b] = (r < rest && c < rest) ? W[(long)(k + nb + r) * ldw + k + nb + c] : T(0);
                    }
                }
                for (int l = 0; l < nb; ++l) {
                    T av[4], bv[4];
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        const int r = r0 + ty * 4 + a;
                        av[a] = r < rest ? P[(nb + r) * (NB + 1) + l] : T(0);
                    }
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const int c = c0 + tx * 4 + b;
                        bv[b] = c < rest ? Us[l * kMaxN + c] : T(0);
                    }
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int b = 0; b < 4; ++b) acc[a][b] = fma(-av[a], bv[b], acc[a][b]);
                }
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const int r = r0 + ty * 4 + a;
                    if (r >= rest) continue;
                    T *row = W + (long)(k + nb + r) * ldw + k + nb;
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const int c = c0 + tx * 4 + b;
                        if (c < rest) row[c] = acc[a][b];
                    }
                }
            }
        __syncthreads();
    }
}

// Inverses of the 32 x 32 diagonal blocks of L (unit lower) and U (upper)
// into Dinv (block b: L^{-1} at Dinv + 2048 b, U^{-1} at Dinv + 2048 b + 1024,
// row-major 32 x 32).  One warp per block, lane = column of the inverse;
// the block is staged in shared memory (buf: 8 x 32 x 33 T).
template <typename T>
__device__ void diag_inverses(int n, const T *W, int ldw, T *Dinv, T *buf) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nbk = (n + 31) / 32;
    T(*blk)[33] = reinterpret_cast<T(*)[33]>(buf + warp * 32 * 33);
    for (int b = warp; b < nbk; b += NT / 32) {
        const int r0 = b * 32, bs = min(32, n - r0);
        for (int i = 0; i < 32; ++i) blk[i][lane] = (i < bs && lane < bs) ? W[(long)(r0 + i) * ldw + r0 + lane] : T(i == lane ? 1 : 0);
        __syncwarp();
        T x[32];
        // unit lower: x_i = delta_ic - sum_{l<i} L_il x_l (c = lane)
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            T s = T(i == lane ? 1 : 0);
#pragma unroll
            for (int l = 0; l < i; ++l) s = fma(-blk[i][l], x[l], s);
            x[i] = s;
        }
        T *Li = Dinv + (long)b * 2048;
#pragma unroll
        for (int i = 0; i < 32; ++i) Li[i * 32 + lane] = x[i];
        // upper: x_i = (delta_ic - sum_{l>i} U_il x_l) / U_ii
#pragma unroll
        for (int i = 31; i >= 0; --i) {
            T s = T(i == lane ? 1 : 0);
#pragma unroll
            for (int l = i + 1; l < 32; ++l) s = fma(-blk[i][l], x[l], s);
            x[i] = s / blk[i][i];
        }
        T *Ui = Li + 1024;
#pragma unroll
        for (int i = 0; i < 32; ++i) Ui[i * 32 + lane] = x[i];
        __syncwarp();
    }
}

// v[c][i] (shared, T) <- U^{-1} L^{-1} v with the factors in W and the
// diagonal-block inverses in Dinv: per 32-row block, y_b = D_b^{-1} v_b
// (thread = (row, rhs)), then the rows after (before) it are updated with
// the block's columns (thread = (row, rhs), 128-byte row segments of W).
template <typename T>
__device__ void lu_solve(int n, int nrhs, const T *W, int ldw, const T *Dinv, T *v, T *tmp) {
    const int tid = threadIdx.x;
    const int nbk = (n + 31) / 32;
    const int r = tid & 31, c = tid >> 5;  // 8 right-hand sides at most
    for (int pass = 0; pass < 2; ++pass) {
        for (int q = 0; q < nbk; ++q) {
            const int b = pass == 0 ? q : nbk - 1 - q;
            const int r0 = b * 32, bs = min(32, n - r0);
            const T *D = Dinv + (long)b * 2048 + (pass == 0 ? 0 : 1024);
            if (c < nrhs && r < bs) {
                const T *drow = D + r * 32;
                T s = T(0);
                if (bs == 32) {  // whole 16-byte pieces of the row, same order
#pragma unroll
                    for (int q = 0; q < 32 / VW16<T>; ++q) {
                        const V16<T> dv = reinterpret_cast<const V16<T> *>(drow)[q];
                        const T *pd = reinterpret_cast<const T *>(&dv);
#pragma unroll
                        for (int e = 0; e < VW16<T>; ++e) s = fma(pd[e], v[c * kMaxN + r0 + q * VW16<T> + e], s);
                    }
                } else {
                    for (int k = 0; k < bs; ++k) s = fma(drow[k], v[c * kMaxN + r0 + k], s);
                }
                tmp[c * 32 + r] = s;
            }
            __syncthreads();
            if (c < nrhs && r < bs) v[c * kMaxN + r0 + r] = tmp[c * 32 + r];
            __syncthreads();
            const int lo = pass == 0 ? r0 + bs : 0, hi = pass == 0 ? n : r0;
            for (int e = tid; e < (hi - lo) * nrhs; e += NT) {
                const int cc = e / (hi - lo), i = lo + e % (hi - lo);
                const T *wr = W + (long)i * ldw + r0;
                T s = v[cc * kMaxN + i];
                if (bs == 32) {  // the row segment in 16-byte pieces (ldw and r0 are multiples of 4)
#pragma unroll
                    for (int q = 0; q < 32 / VW16<T>; ++q) {
                        const V16<T> wv = reinterpret_cast<const V16<T> *>(wr)[q];
                        const T *pw = reinterpret_cast<const T *>(&wv);
#pragma unroll
                        for (int e = 0; e < VW16<T>; ++e) s = fma(-pw[e], v[cc * kMaxN + r0 + q * VW16<T> + e], s);
                    }
                } else {
                    for (int j = 0; j < bs; ++j) s = fma(-wr[j], v[cc * kMaxN + r0 + j], s);
                }
                v[cc * kMaxN + i] = s;
            }
            __syncthreads();
        }
    }
}

// r = b - A x (FP64) for the thread's rows i = tid and tid + NT (n <= 2 NT),
// products in column order per row, 16 columns per batch with both rows'
// loads in flight; rloc[c], xloc[c] receive the thread's max |r_c| and |x_c|.
// NR >= nrhs bounds the unrolled right-hand-side loops.
template <int NR>
__device__ __forceinline__ void residual_rows(const BatchSys &d, int n, int nrhs, const double *xs, double *rloc,
                                              double *xloc) {
    const int i0 = threadIdx.x, i1 = threadIdx.x + NT;
    const bool v0 = i0 < n, v1 = i1 < n;
    double acc0[NR], acc1[NR];
#pragma unroll
    for (int c = 0; c < NR; ++c) { acc0[c] = 0.0; acc1[c] = 0.0; }
    const double *a0p = d.A + i0, *a1p = d.A + i1;
    int j = 0;
    for (; j + 16 <= n; j += 16) {
        double a0[16], a1[16];
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            a0[t] = v0 ? a0p[(long)(j + t) * d.lda] : 0.0;
            a1[t] = v1 ? a1p[(long)(j + t) * d.lda] : 0.0;
        }
#pragma unroll
        for (int t = 0; t < 16; ++t)
#pragma unroll
            for (int c = 0; c < NR; ++c)
                if (c < nrhs) {
                    const double x = xs[c * kMaxN + j + t];
                    acc0[c] = fma(a0[t], x, acc0[c]);
                    acc1[c] = fma(a1[t], x, acc1[c]);
                }
    }
    for (; j < n; ++j) {
        const double a0 = v0 ? a0p[(long)j * d.lda] : 0.0, a1 = v1 ? a1p[(long)j * d.lda] : 0.0;
#pragma unroll
        for (int c = 0; c < NR; ++c)
            if (c < nrhs) {
                const double x = xs[c * kMaxN + j];
                acc0[c] = fma(a0, x, acc0[c]);
                acc1[c] = fma(a1, x, acc1[c]);
            }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int i = h ? i1 : i0;
        if (i >= n) continue;
#pragma unroll
        for (int c = 0; c < NR; ++c)
            if (c < nrhs) {
                const double r = d.B[(long)c * d.ldb + i] - (h ? acc1[c] : acc0[c]);
                d.R[(long)c * n + i] = r;
                rloc[c] = fmax(rloc[c], (r == r) ? fabs(r) : INFINITY);
                xloc[c] = fmax(xloc[c], fabs(xs[c * kMaxN + i]));
            }
    }
}

template <typename T>
__global__ void __launch_bounds__(NT, 2)
batched_kernel(BatchSys *__restrict__ sys, const int *__restrict__ order, int count, int *counter, int prec,
               int itermax, double tol, double stall_ratio) {
    constexpr int NB = BCfg<T>::NB;
    extern __shared__ __align__(16) unsigned char raw[];
    T *P = reinterpret_cast<T *>(raw);
    T *Us = P + (size_t)kMaxN * (NB + 1);
    double *xs = reinterpret_cast<double *>(Us + (size_t)NB * kMaxN);
    Shared &sh = *reinterpret_cast<Shared *>(xs + (size_t)kMaxN * kMaxRhs);
    const int tid = threadIdx.x;
    const double u64 = 1.1102230246251565e-16;
    for (;;) {
        if (tid == 0) {
            const int q = atomicAdd(counter, 1);
            sh.sys = q < count ? order[q] : -1;
        }
        __syncthreads();
        const int id = sh.sys;
        if (id < 0) break;
        BatchSys &d = sys[id];
        const int n = d.n, nrhs = d.nrhs, ldw = d.ldw;
        T *W = static_cast<T *>(d.W);
        if (tid == 0) { sh.flags = 0; sh.info = 0; sh.stop = 0; }
        for (int i = tid; i < n; i += NT) d.perm[i] = i;
        __syncthreads();
        // ---- convert: row sums of |A| (fixed order per row), W = fl(A) through the panel buffer
        // A is read once: column chunks of NB through the panel buffer, rows
        // fixed per thread (tid, tid + NT) with the chunk's loads in flight,
        // and the row sums of |A| taken from the same values in column order
        double rsum[2] = {0.0, 0.0};
        for (int c0 = 0; c0 < n; c0 += NB) {
            const int w = min(NB, n - c0);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int i = tid + h * NT;
                if (i < n) {
                    const double *ai = d.A + (long)c0 * d.lda + i;
                    double a[NB];
#pragma unroll
                    for (int j = 0; j < NB; ++j) a[j] = j < w ? __ldcs(ai + (long)j * d.lda) : 0.0;
                    double sacc = rsum[h];
#pragma unroll
                    for (int j = 0; j < NB; ++j)
                        if (j < w) {
                            sacc += fabs(a[j]);
                            P[i * (NB + 1) + j] = (T)a[j];
                        }
                    rsum[h] = sacc;
                }
            }
            __syncthreads();
            for (int e = tid; e < n * w; e += NT) {
                const int i = e / w, j = e % w;
                W[(long)i * ldw + c0 + j] = P[i * (NB + 1) + j];
            }
            __syncthreads();
        }
        bool bad = false;
        double rmax = 0.0;
#pragma unroll
        for (int h = 0; h < 2; ++h)
            if (tid + h * NT < n) {
                if (!(rsum[h] <= 1.79769313486231570815e308)) bad = true;
                rmax = fmax(rmax, rsum[h]);
            }
        const double an = block_max(bad ? __longlong_as_double(0x7ff0000000000000LL) : rmax, sh);
        for (int c = 0; c < nrhs; ++c) {
            double m = 0.0;
            for (int i = tid; i < n; i += NT) m = fmax(m, fabs(d.B[(long)c * d.ldb + i]));
            m = block_max(m, sh);
            if (tid == 0) sh.bnorm[c] = m;
        }
        if (tid == 0) {
            sh.anorm = an;
            if (!(an <= 1.79769313486231570815e308)) sh.flags |= MP_FLAG_NONFINITE_INPUT;
            for (int c = 0; c < nrhs; ++c)
                if (!(sh.bnorm[c] <= 1.79769313486231570815e308)) sh.flags |= MP_FLAG_NONFINITE_INPUT;
        }
        __syncthreads();
        if (sh.flags & MP_FLAG_NONFINITE_INPUT) {
            if (tid == 0) { d.flags = sh.flags; d.iter = 0; d.info = 0; d.bwd = INFINITY; }
            __syncthreads();
            continue;
        }
        // ---- factor
        if constexpr (sizeof(T) == 4) {  // the panel width the schedule gave this system
            if (d.nb == 8) lu_factor<T, 8>(d, W, ldw, P, Us, sh, prec);
            else lu_factor<T, NB>(d, W, ldw, P, Us, sh, prec);  // the buffers' width bounds the panel
        } else {
            lu_factor<T, NB>(d, W, ldw, P, Us, sh, prec);
        }
        if (sh.flags & MP_FLAG_LOWP_BREAKDOWN) {
            if (tid == 0) { d.flags = sh.flags; d.iter = 0; d.info = sh.info; d.bwd = INFINITY; }
            __syncthreads();
            continue;
        }
        // ---- diagonal-block inverses for the solves (panel buffer as scratch)
        T *Dinv = static_cast<T *>(d.Dinv);
        diag_inverses<T>(n, W, ldw, Dinv, P);
        __syncthreads();
        // ---- x0 = M b, then the refinement loop (steps 4-7)
        T *v = Us;  // nrhs x kMaxN vectors
        T *tmp = P;  // 8 x 32 scratch of the solves
        for (int e = tid; e < n * nrhs; e += NT) {
            const int c = e / n, i = e % n;
            v[c * kMaxN + i] = (T)(d.B[(long)c * d.ldb + d.perm[i]] / pow2_ceil_d(sh.bnorm[c]));
        }
        __syncthreads();
        lu_solve<T>(n, nrhs, W, ldw, Dinv, v, tmp);
        for (int e = tid; e < n * nrhs; e += NT) {
            const int c = e / n, i = e % n;
            const double z = (double)v[c * kMaxN + i] * pow2_ceil_d(sh.bnorm[c]);
            d.X[(long)c * d.ldx + i] = z;
        }
        if (tid < kMaxRhs) { sh.zprev[tid] = 0.0; sh.znorm[tid] = 0.0; }
        __syncthreads();
        int it = 0;
        bool conv = false;
        double worst = 0.0;
        for (;;) {
            // x into shared memory, r = b - A x in FP64 (row per thread, j in order)
            for (int e = tid; e < n * nrhs; e += NT) {
                const int c = e / n, i = e % n;
                xs[c * kMaxN + i] = d.X[(long)c * d.ldx + i];
            }
            __syncthreads();
            double rloc[kMaxRhs], xloc[kMaxRhs];
#pragma unroll
            for (int c = 0; c < kMaxRhs; ++c) { rloc[c] = 0.0; xloc[c] = 0.0; }
            if (nrhs <= 1) residual_rows<1>(d, n, nrhs, xs, rloc, xloc);
            else if (nrhs <= 2) residual_rows<2>(d, n, nrhs, xs, rloc, xloc);
            else if (nrhs <= 4) residual_rows<4>(d, n, nrhs, xs, rloc, xloc);
            else residual_rows<8>(d, n, nrhs, xs, rloc, xloc);
            for (int c = 0; c < nrhs; ++c) {
                const double rm = block_max(rloc[c], sh);
                const double xm = block_max(xloc[c], sh);
                if (tid == 0) { sh.rnorm[c] = rm; sh.xnorm[c] = xm; }
            }
            __syncthreads();
            if (tid == 0) {
                bool done = true, nonfinite = false, stalled = false, all_tol = true;
                worst = 0.0;
                for (int c = 0; c < nrhs; ++c) {
                    const double den = sh.anorm * sh.xnorm[c] + sh.bnorm[c];
                    double b = den > 0.0 ? sh.rnorm[c] / den : (sh.rnorm[c] > 0.0 ? INFINITY : 0.0);
                    if (!(sh.rnorm[c] == sh.rnorm[c])) b = INFINITY;
                    const bool stagnant = it >= 2 && sh.znorm[c] > stall_ratio * sh.zprev[c];
                    const bool at_floor =
                        b == 0.0 || b <= 2.0 * u64 || sh.znorm[c] <= 4.0 * u64 * sh.xnorm[c] || stagnant;
                    if (!(b <= tol)) all_tol = false;
                    if (!(b <= tol && at_floor)) done = false;
                    if (!(b <= tol) && stagnant) stalled = true;
                    if (!(b < INFINITY)) nonfinite = true;
                    worst = fmax(worst, b);
                }
                int stop = 0;
                if (nonfinite) { sh.flags |= MP_FLAG_LOWP_BREAKDOWN; stop = 1; }
                else if (done) { conv = true; stop = 1; }
                else if (stalled) { sh.flags |= MP_FLAG_STALLED; stop = 1; }
                else if (it >= itermax) { conv = all_tol; stop = 1; }
                sh.stop = stop | (conv ? 2 : 0);
                d.bwd = worst;
                for (int c = 0; c < nrhs; ++c) { sh.zprev[c] = sh.znorm[c]; sh.znorm[c] = 0.0; }
            }
            __syncthreads();
            if (sh.stop & 1) { conv = (sh.stop & 2) != 0; break; }
            // z = M (r / s), x += s z
            for (int e = tid; e < n * nrhs; e += NT) {
                const int c = e / n, i = e % n;
                v[c * kMaxN + i] = (T)(d.R[(long)c * n + d.perm[i]] / pow2_ceil_d(sh.rnorm[c]));
            }
            __syncthreads();
            lu_solve<T>(n, nrhs, W, ldw, Dinv, v, tmp);
            for (int c = 0; c < nrhs; ++c) {
                const double s = pow2_ceil_d(sh.rnorm[c]);
                double zm = 0.0;
                for (int i = tid; i < n; i += NT) {
                    const double z = (double)v[c * kMaxN + i] * s;
                    d.X[(long)c * d.ldx + i] += z;
                    zm = fmax(zm, (z == z) ? fabs(z) : INFINITY);
                }
                zm = block_max(zm, sh);
                if (tid == 0) sh.znorm[c] = zm;
            }
            __syncthreads();
            ++it;
        }
        if (tid == 0) {
            d.iter = it;
            d.info = 0;
            d.flags = sh.flags | (conv ? 0u : 0x80000000u);  // high bit: needs the fallback pass
        }
        __syncthreads();
    }
}

size_t carve_b(size_t &off, size_t bytes) {
    off = (off + 255) / 256 * 256;
    const size_t at = off;
    off += bytes;
    return at;
}

template <typename T>
cudaError_t launch_batched(BatchSys *dsys, const int *dorder, int count, int *dcounter, int prec, int itermax,
                           double tol, double stall_ratio, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    const size_t smem = batched_smem_bytes<T>();
    auto kern = batched_kernel<T>;
    cudaError_t e = mp_smem_attr(kern, smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
    if (e != cudaSuccess) return e;
    const int grid = std::min(count, std::max(sms, 1) * std::max(per_sm, 1));
    e = cudaMemsetAsync(dcounter, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    mp_note_launch();
    kern<<<grid, NT, smem, s>>>(dsys, dorder, count, dcounter, prec, itermax, tol, stall_ratio);
    return cudaGetLastError();
}

}  // namespace

size_t batched_layout(int batch, const int *n, const int *nrhs, bool fp64, size_t *per_sys_off) {
    size_t off = 0;
    carve_b(off, sizeof(BatchSys) * (size_t)batch);
    carve_b(off, sizeof(int) * (size_t)batch * 2);
    carve_b(off, sizeof(int) * 4);
    const size_t el = fp64 ? sizeof(double) : sizeof(float);
    for (int b = 0; b < batch; ++b) {
        const int nn = std::max(n[b], 1), rr = std::max(nrhs[b], 1);
        const size_t ldw = (size_t)(nn + 3) / 4 * 4;
        const size_t at = carve_b(off, el * (size_t)nn * ldw);
        carve_b(off, sizeof(double) * (size_t)nn * rr);
        carve_b(off, sizeof(int) * (size_t)nn);
        carve_b(off, el * 2048 * (size_t)((nn + 31) / 32));
        if (per_sys_off) per_sys_off[b] = at;
    }
    return (off + 255) / 256 * 256;
}

// The active schedule: the compiled-in table unless mp_batched_set_schedule
// replaced it (process-wide).
namespace {
std::mutex g_sched_mu;
std::vector<int> g_sched_nmax(kBatchedNmax, kBatchedNmax + kBatchedRanges);
std::vector<int> g_sched_nb(kBatchedNb, kBatchedNb + kBatchedRanges);
int schedule_nb(int n) {
    std::lock_guard<std::mutex> g(g_sched_mu);
    for (size_t i = 0; i < g_sched_nmax.size(); ++i)
        if (n <= g_sched_nmax[i]) return g_sched_nb[i];
    return 16;
}
}  // namespace

extern "C" int mp_batched_set_schedule(int count, const int *nmax, const int *nb) {
    if (count < 0 || count > 64) return mp_arg_fail(1, "count must be in [0, 64]");
    std::lock_guard<std::mutex> g(g_sched_mu);
    if (count == 0) {
        g_sched_nmax.assign(kBatchedNmax, kBatchedNmax + kBatchedRanges);
        g_sched_nb.assign(kBatchedNb, kBatchedNb + kBatchedRanges);
        return 0;
    }
    if (!nmax) return mp_arg_fail(2, "nmax is NULL");
    if (!nb) return mp_arg_fail(3, "nb is NULL");
    for (int i = 0; i < count; ++i) {
        if (nmax[i] < 1 || (i > 0 && nmax[i] <= nmax[i - 1])) return mp_arg_fail(2, "nmax must increase");
        if (nb[i] != 8 && nb[i] != 16) return mp_arg_fail(3, "nb must be 8 or 16");
    }
    if (nmax[count - 1] < MP_BATCH_MAX_N) return mp_arg_fail(2, "the last range must reach MP_BATCH_MAX_N");
    g_sched_nmax.assign(nmax, nmax + count);
    g_sched_nb.assign(nb, nb + count);
    return 0;
}

extern "C" int mp_batched_get_schedule(int cap, int *count, int *nmax, int *nb) {
    std::lock_guard<std::mutex> g(g_sched_mu);
    if (count) *count = (int)g_sched_nmax.size();
    for (int i = 0; i < (int)g_sched_nmax.size() && i < cap; ++i) {
        if (nmax) nmax[i] = g_sched_nmax[i];
        if (nb) nb[i] = g_sched_nb[i];
    }
    return 0;
}

int batched_run(int batch, const int *n, const int *nrhs, const double *const *A, const int *lda,
                const double *const *B, const int *ldb, double *const *X, const int *ldx, int32_t *const *ipiv,
                int *iter, unsigned *flags, int *info, void *work, const mp_opts &o, cudaStream_t s,
                cudaError_t *cerr) {
    *cerr = cudaSuccess;
    const bool fb = o.allow_fallback != 0;
    std::vector<size_t> soff(batch);
    batched_layout(batch, n, nrhs, fb, soff.data());
    char *base = static_cast<char *>(work);
    size_t off = 0;
    BatchSys *dsys = reinterpret_cast<BatchSys *>(base + carve_b(off, sizeof(BatchSys) * (size_t)batch));
    int *dorder = reinterpret_cast<int *>(base + carve_b(off, sizeof(int) * (size_t)batch * 2));
    int *dcounter = reinterpret_cast<int *>(base + carve_b(off, sizeof(int) * 4));
    std::vector<BatchSys> hs(batch);
    const size_t el = fb ? sizeof(double) : sizeof(float);
    for (int b = 0; b < batch; ++b) {
        BatchSys &d = hs[b];
        std::memset(&d, 0, sizeof d);
        const int nn = std::max(n[b], 1);
        d.n = n[b];
        d.nrhs = nrhs[b];
        d.lda = lda[b];
        d.ldb = ldb[b];
        d.ldx = ldx[b];
        d.ldw = (nn + 3) / 4 * 4;
        d.nb = schedule_nb(nn);
        d.A = A[b];
        d.B = B[b];
        d.X = X[b];
        d.ipiv = ipiv[b];
        char *p = base + soff[b];
        d.W = p;
        size_t o2 = soff[b] + el * (size_t)nn * d.ldw;
        o2 = (o2 + 255) / 256 * 256;
        d.R = reinterpret_cast<double *>(base + o2);
        o2 += sizeof(double) * (size_t)nn * std::max(nrhs[b], 1);
        o2 = (o2 + 255) / 256 * 256;
        d.perm = reinterpret_cast<int *>(base + o2);
        o2 += sizeof(int) * (size_t)nn;
        o2 = (o2 + 255) / 256 * 256;
        d.Dinv = base + o2;
    }
    // queue: non-empty systems by decreasing n^3 (longest first)
    std::vector<int> ord;
    for (int b = 0; b < batch; ++b)
        if (n[b] > 0 && nrhs[b] > 0) ord.push_back(b);
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return n[a] > n[b]; });
    auto fail = [&](cudaError_t e) { *cerr = e; return -1; };
    cudaError_t e;
    if ((e = cudaMemcpyAsync(dsys, hs.data(), sizeof(BatchSys) * (size_t)batch, cudaMemcpyHostToDevice, s)))
        return fail(e);
    if (!ord.empty() &&
        (e = cudaMemcpyAsync(dorder, ord.data(), sizeof(int) * ord.size(), cudaMemcpyHostToDevice, s)))
        return fail(e);
    if ((e = launch_batched<float>(dsys, dorder, (int)ord.size(), dcounter, o.prec, o.itermax, o.tol, o.stall_ratio, s)))
        return fail(e);
    if ((e = cudaMemcpyAsync(hs.data(), dsys, sizeof(BatchSys) * (size_t)batch, cudaMemcpyDeviceToHost, s)))
        return fail(e);
    if ((e = cudaStreamSynchronize(s))) return fail(e);
    std::vector<int> redo;
    for (int b : ord)
        if ((hs[b].flags & 0x80000000u) || (hs[b].flags & MP_FLAG_LOWP_BREAKDOWN))
            if (!(hs[b].flags & MP_FLAG_NONFINITE_INPUT)) redo.push_back(b);
    std::vector<int> low_iter(batch, 0);
    std::vector<unsigned> low_flags(batch, 0u);
    for (int b = 0; b < batch; ++b) { low_iter[b] = hs[b].iter; low_flags[b] = hs[b].flags & 0x7fffffffu; }
    if (!redo.empty() && fb) {
        if ((e = cudaMemcpyAsync(dorder, redo.data(), sizeof(int) * redo.size(), cudaMemcpyHostToDevice, s)))
            return fail(e);
        if ((e = launch_batched<double>(dsys, dorder, (int)redo.size(), dcounter, MP_PREC_FP32, 5, o.tol, o.stall_ratio,
                                        s)))
            return fail(e);
        if ((e = cudaMemcpyAsync(hs.data(), dsys, sizeof(BatchSys) * (size_t)batch, cudaMemcpyDeviceToHost, s)))
            return fail(e);
        if ((e = cudaStreamSynchronize(s))) return fail(e);
    }
    for (int b = 0; b < batch; ++b) {
        const bool was_redo = std::find(redo.begin(), redo.end(), b) != redo.end();
        unsigned f = low_flags[b] & ~0x80000000u;
        int it = low_iter[b], inf = 0;
        if (was_redo && fb) {
            f |= MP_FLAG_FALLBACK;
            it = -1;
            inf = hs[b].info;
        } else if (was_redo) {
            f |= MP_FLAG_NOT_CONVERGED;
        }
        if (iter) iter[b] = it;
        if (flags) flags[b] = f;
        if (info) info[b] = inf;
    }
    return 0;
}

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" size_t mp_gesv_batched_workspace_bytes(int batch, const int *n, const int *nrhs, const mp_opts *opts) {
    mp_opts o;
    if (opts) o = *opts; else mp_default_opts(&o);
    if (batch < 0 || (batch > 0 && (!n || !nrhs))) return 0;
    for (int b = 0; b < batch; ++b)
        if (n[b] < 0 || nrhs[b] < 0) return 0;
    return batched_layout(batch, n, nrhs, o.allow_fallback != 0, nullptr);
}

extern "C" int mp_gesv_batched(int batch, const int *n, const int *nrhs, const double *const *A, const int *lda,
                               const double *const *B, const int *ldb, double *const *X, const int *ldx,
                               int32_t *const *ipiv, int *iter, unsigned *flags, int *info, void *work,
                               size_t work_bytes, const mp_opts *opts, void *stream) {
    mp_opts o;
    if (opts) o = *opts; else mp_default_opts(&o);
    if (batch < 0) return mp_arg_fail(1, "batch < 0");
    if (batch == 0) return 0;
    if (!n) return mp_arg_fail(2, "n is NULL");
    if (!nrhs) return mp_arg_fail(3, "nrhs is NULL");
    if (!A || !lda) return mp_arg_fail(4, "A or lda is NULL");
    if (!B || !ldb) return mp_arg_fail(6, "B or ldb is NULL");
    if (!X || !ldx) return mp_arg_fail(8, "X or ldx is NULL");
    if (!ipiv) return mp_arg_fail(10, "ipiv is NULL");
    for (int b = 0; b < batch; ++b) {
        if (n[b] < 0 || n[b] > MP_BATCH_MAX_N) return mp_arg_fail(2, "n[i] must be in [0, MP_BATCH_MAX_N]");
        if (nrhs[b] < 0 || nrhs[b] > 8) return mp_arg_fail(3, "nrhs[i] must be in [0, 8]");
        if (n[b] == 0 || nrhs[b] == 0) continue;
        if (!A[b] || lda[b] < n[b]) return mp_arg_fail(5, "A[i] NULL or lda[i] < n[i]");
        if (!B[b] || ldb[b] < n[b]) return mp_arg_fail(7, "B[i] NULL or ldb[i] < n[i]");
        if (!X[b] || ldx[b] < n[b]) return mp_arg_fail(9, "X[i] NULL or ldx[i] < n[i]");
        if (!ipiv[b]) return mp_arg_fail(10, "ipiv[i] is NULL");
    }
    if (o.prec != MP_PREC_FP32 && o.prec != MP_PREC_BF16 && o.prec != MP_PREC_FP16)
        return mp_arg_fail(16, "batched solve supports prec FP32, BF16, FP16");
    if (o.itermax < 0 || !(o.tol > 0.0) || !(o.stall_ratio > 0.0)) return mp_arg_fail(16, "invalid options");
    if (!work) return mp_arg_fail(14, "workspace is NULL");
    if (work_bytes < batched_layout(batch, n, nrhs, o.allow_fallback != 0, nullptr))
        return mp_arg_fail(15, "workspace too small");
    cudaError_t ce;
    const int r = batched_run(batch, n, nrhs, A, lda, B, ldb, X, ldx, ipiv, iter, flags, info, work, o,
                              static_cast<cudaStream_t>(stream), &ce);
    if (r) return mp_cuda_fail(ce, "batched solve", __FILE__, __LINE__);
    return 0;
}
