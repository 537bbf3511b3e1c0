// blas3.cu -- row exchanges, SIMT GEMM update and small triangular solves
// used inside the blocked factorization (Section 3.1.1: the SGETRF building
// blocks; Section 2.1: PA = LU).  All matrices are row-major.
#include <algorithm>
#include <climits>
#include <mutex>
#include <type_traits>

#include "common.cuh"
#include "kernels.cuh"

// ============================================================================
// Row exchanges.  A run of LAPACK-style swaps (row k <-> row ipiv[k]-1, in
// order) is first composed into a list of (destination, source) row moves,
// then every column range is permuted with one gather/scatter through shared
// memory.  Rows are contiguous in the row-major W, so each move copies whole
// 128-byte row segments.
// ============================================================================
namespace {

constexpr int kComposeThreads = 1024;
constexpr int kComposeSmemRows = 40960;  // 160 KB map in shared memory

__global__ void __launch_bounds__(kComposeThreads)
compose_swaps_kernel(const int32_t *__restrict__ ipiv, int k1, int k2, int n, int2 *pairs,
                     int *npairs, int *gmap) {
    extern __shared__ int dyn[];
    const int npiv = k2 - k1;
    const int rows = n - k1;
    int *piv = dyn;                       // npiv
    const bool use_smem = rows <= kComposeSmemRows;
    int *map = use_smem ? dyn + npiv : gmap + k1;  // map[i - k1] = source row now at row i
    __shared__ int count;
    const int tid = threadIdx.x;
    if (tid == 0) count = 0;
    for (int t = tid; t < npiv; t += blockDim.x) piv[t] = ipiv[k1 + t] - 1;
    if (use_smem)
        for (int t = tid; t < rows; t += blockDim.x) map[t] = k1 + t;
    __syncthreads();
    if (tid == 0) {
        for (int t = 0; t < npiv; ++t) {
            const int k = k1 + t, p = piv[t];
            if (p != k && p >= k && p < n) {
                const int a = map[k - k1];
                map[k - k1] = map[p - k1];
                map[p - k1] = a;
            }
        }
    }
    __syncthreads();
    // rows of the block itself
    for (int t = tid; t < npiv; t += blockDim.x) {
        const int row = k1 + t;
        const int src = map[t];
        if (src != row) {
            const int slot = atomicAdd(&count, 1);
            pairs[slot] = make_int2(row, src);
        }
    }
    __syncthreads();
    // pivot rows below the block (deduplicated through the map itself)
    for (int t = tid; t < npiv; t += blockDim.x) {
        const int p = piv[t];
        if (p >= k2 && p < n) {
            const int src = atomicExch(&map[p - k1], INT_MIN);
            if (src != INT_MIN && src != p) {
                const int slot = atomicAdd(&count, 1);
                pairs[slot] = make_int2(p, src);
            }
        }
    }
    __syncthreads();
    if (!use_smem) {  // restore the identity for the rows we touched
        for (int t = tid; t < npiv; t += blockDim.x) {
            map[t] = k1 + t;
            const int p = piv[t];
            if (p >= k2 && p < n) map[p - k1] = p;
        }
    }
    if (tid == 0) *npairs = count;
}

template <typename T, int CW>
__global__ void __launch_bounds__(256)
apply_moves_kernel(T *__restrict__ W, long ld, const int2 *__restrict__ pairs,
                   const int *__restrict__ npairs, int c0, int c1, int c2, int c3, int *perm) {
    extern __shared__ unsigned char dyn_raw[];
    T *tile = reinterpret_cast<T *>(dyn_raw);
    const int np = *npairs;
    if (np == 0) return;
    if (perm && blockIdx.x == gridDim.x - 1) {  // the last CTA also permutes perm
        int *pv = reinterpret_cast<int *>(tile);
        for (int t = threadIdx.x; t < np; t += blockDim.x) pv[t] = perm[pairs[t].y];
        __syncthreads();
        for (int t = threadIdx.x; t < np; t += blockDim.x) perm[pairs[t].x] = pv[t];
        __syncthreads();
    }
    const int nch1 = (c1 - c0 + CW - 1) / CW;
    int cs, ce;
    if ((int)blockIdx.x < nch1) {
        cs = c0 + blockIdx.x * CW;
        ce = min(cs + CW, c1);
    } else {
        cs = c2 + (blockIdx.x - nch1) * CW;
        ce = min(cs + CW, c3);
    }
    const int w = ce - cs;
    if (w <= 0) return;
    for (int idx = threadIdx.x; idx < np * CW; idx += blockDim.x) {
        const int pr = idx / CW, cc = idx - pr * CW;
        if (cc < w) tile[idx] = W[(long)pairs[pr].y * ld + cs + cc];
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < np * CW; idx += blockDim.x) {
        const int pr = idx / CW, cc = idx - pr * CW;
        if (cc < w) W[(long)pairs[pr].x * ld + cs + cc] = tile[idx];
    }
}

// One leaf step of the panel factorization, after the leaf (columns
// [k, k+kb)) has been factored:
//   U = X A12, X = L11^{-1} from the panel kernel
//                     (A12: rows k..k+kb of the columns [k+kb+coff, k+kb+coff+N))
//   A22 -= L21 U      (rows [k+kb, k+kb+M) of the same columns)
// over (TR-row tile, 128-column chunk) pairs.  Columns of U are independent,
// so every tile forms the U columns of its chunk in shared memory (the same
// arithmetic in each, so all copies agree bit for bit) and updates its
// TR x 128 tile of A22 with FP32 (FP64) FMAs in the order l = 0..kb-1.
//
// Two forms.  (a) After the leaf's row exchange: one CTA per tile.  (b)
// Persistent, with the exchange folded in: A12 rows are read from the rows
// the moves bring there, tiles skip the moved rows of A22, and the tile that
// draws the last ticket of its chunk computes the moved rows (source row -
// L21 U) into shared memory and stores them.  Every write that another tile
// of the chunk could still read (U over A12, the moved rows) is made by that
// last tile, after every tile of the chunk has finished reading.  No CTA waits
// for another.
constexpr int kLeafTileCols = 128;
// dynamic shared memory of the persistent form: a staging area (moved rows,
// exchange tiles) and a bitmap of the moved rows of A22; more than half of an
// SM's shared memory, so that it runs at one CTA per SM
constexpr int kLeafStageBytes = 40 * 1024;
inline size_t leaf_update_pad_bytes() { return 120 * 1024; }
constexpr int kLeafMaxBitmapRows = (120 - 40) * 1024 * 8;

template <typename T, int KBMAX, int TR>
struct LeafSmem {
    __align__(16) T Us[KBMAX][kLeafTileCols];
    T Ls[KBMAX][KBMAX + 1];  // X = L11^{-1} (unit lower)
    T Lt[TR][KBMAX + 1];
    int a12[KBMAX];          // row that A12 row i is read from
    int2 mv[2 * KBMAX];      // moved rows of A22: (destination, source)
    int nmv;
    bool last;
};

// One (TR-row tile, chunk) of the leaf step; R = row tiles per chunk.
// MOVES: the persistent form (b), with bits = moved rows of A22 (bit r: row
// k+kb+r) and stage = kLeafStageBytes of shared memory.
template <typename T, int KBMAX, int TR, bool MOVES>
__device__ __forceinline__ void leaf_tile(LeafSmem<T, KBMAX, TR> &sm, T *W, long ld, int k, int kb, int coff, int N,
                                          int M, unsigned *tickets, int r0, int chunk, int R, const unsigned *bits,
                                          T *stage) {
    constexpr int NTHR = TR * 4, NG = NTHR / kLeafTileCols;
    const int tid = threadIdx.x;
    const int c0 = chunk * kLeafTileCols;
    const int w = min(kLeafTileCols, N - c0);
    const int cb = k + kb + coff + c0;  // first column of the chunk
    for (int idx = tid; idx < kb * kLeafTileCols; idx += NTHR) {
        const int i = idx / kLeafTileCols, c = idx - i * kLeafTileCols;
        const int row = MOVES ? sm.a12[i] : k + i;
        sm.Us[i][c] = c < w ? W[(long)row * ld + cb + c] : T(0);
    }
    for (int idx = tid; idx < TR * kb; idx += NTHR) {
        const int r = idx / kb, l = idx - r * kb;
        sm.Lt[r][l] = r0 + r < M ? W[(long)(k + kb + r0 + r) * ld + k + l] : T(0);
    }
    // this thread's 8 rows x 4 columns of the A22 tile (16-byte vectors when
    // the 4 columns are inside the tile: the tile starts on a multiple of 4
    // columns and ld is a multiple of 32; rows the leaf's moves replace are
    // read but never stored).  The persistent form (one CTA per SM, nothing
    // else to hide latency) loads them before the U computation.
    using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
    constexpr int VW = 16 / sizeof(T);
    const int ty = tid >> 5, tx = tid & 31;
    const bool full4 = tx * 4 + 3 < w;
    const int rows = M - (r0 + ty * 8);  // rows of this thread's 8 inside A22
    T *const tile = W + (long)(k + kb + r0 + ty * 8) * ld + (cb + tx * 4);
    T acc[8][4];
    auto load_tile = [&]() {
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            const T *src = tile + (long)a * ld;
            if (a < rows && full4) {
#pragma unroll
                for (int q = 0; q < 4 / VW; ++q) {
                    const V v = reinterpret_cast<const V *>(src)[q];
                    const T *pv = reinterpret_cast<const T *>(&v);
#pragma unroll
                    for (int e = 0; e < VW; ++e) acc[a][q * VW + e] = pv[e];
                }
            } else {
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = (a < rows && tx * 4 + b < w) ? src[b] : T(0);
            }
        }
    };
    if constexpr (MOVES) load_tile();
    __syncthreads();
    // U = X A12 for the chunk's columns: thread (g, c) forms rows g, g+NG, ...
    // of column c (independent dot products, l in order)
    {
        const int c = tid & (kLeafTileCols - 1), g = tid / kLeafTileCols;
        T u[(KBMAX + NG - 1) / NG];
#pragma unroll
        for (int q = 0; q < (KBMAX + NG - 1) / NG; ++q) {
            const int i = g + NG * q;
            T v = i < kb ? sm.Us[i][c] : T(0);
            for (int l = 0; l < i; ++l) v = fma(sm.Ls[i][l], sm.Us[l][c], v);
            u[q] = v;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < (KBMAX + NG - 1) / NG; ++q) {
            const int i = g + NG * q;
            if (i < kb) sm.Us[i][c] = u[q];
        }
    }
    __syncthreads();
    {
        if constexpr (!MOVES) load_tile();
        for (int l = 0; l < kb; ++l) {
            T bv[4], av[8];
#pragma unroll
            for (int q = 0; q < 4 / VW; ++q) {
                const V v = reinterpret_cast<const V *>(&sm.Us[l][tx * 4])[q];
                const T *pv = reinterpret_cast<const T *>(&v);
#pragma unroll
                for (int e = 0; e < VW; ++e) bv[q * VW + e] = pv[e];
            }
#pragma unroll
            for (int a = 0; a < 8; ++a) av[a] = sm.Lt[ty * 8 + a][l];
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fma(-av[a], bv[b], acc[a][b]);
        }
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            if (a >= rows) continue;
            if (MOVES) {
                const int rr = r0 + ty * 8 + a;
                if ((bits[rr >> 5] >> (rr & 31)) & 1u) continue;  // a moved row: the last tile stores it
            }
            T *dst = tile + (long)a * ld;
            if (full4) {
#pragma unroll
                for (int q = 0; q < 4 / VW; ++q) {
                    V v;
                    T *pv = reinterpret_cast<T *>(&v);
#pragma unroll
                    for (int e = 0; e < VW; ++e) pv[e] = acc[a][q * VW + e];
                    reinterpret_cast<V *>(dst)[q] = v;
                }
            } else {
#pragma unroll
                for (int b = 0; b < 4; ++b)
                    if (tx * 4 + b < w) dst[b] = acc[a][b];
            }
        }
    }
    // every read of A12 (and of the moved rows' sources) in this tile is done
    __threadfence();
    __syncthreads();
    if (tid == 0) sm.last = atomicAdd(&tickets[chunk], 1u) == (unsigned)R - 1;
    __syncthreads();
    if (!sm.last) return;
    __threadfence();
    if (MOVES) {  // moved rows d of A22: W[src] - L21[d] U, staged before any store
        for (int idx = tid; idx < sm.nmv * kLeafTileCols; idx += NTHR) {
            const int j = idx / kLeafTileCols, c = idx - j * kLeafTileCols;
            if (c >= w) continue;
            const int2 mv = sm.mv[j];
            T v = W[(long)mv.y * ld + cb + c];
            const T *lrow = W + (long)mv.x * ld + k;
            for (int l = 0; l < kb; ++l) v = fma(-lrow[l], sm.Us[l][c], v);
            stage[idx] = v;
        }
        __syncthreads();
    }
    for (int idx = tid; idx < kb * kLeafTileCols; idx += NTHR) {
        const int i = idx / kLeafTileCols, c = idx - i * kLeafTileCols;
        if (c < w) W[(long)(k + i) * ld + cb + c] = sm.Us[i][c];
    }
    if (MOVES)
        for (int idx = tid; idx < sm.nmv * kLeafTileCols; idx += NTHR) {
            const int j = idx / kLeafTileCols, c = idx - j * kLeafTileCols;
            if (c < w) W[(long)sm.mv[j].x * ld + cb + c] = stage[idx];
        }
    if (tid == 0) tickets[chunk] = 0u;
}

template <typename T, int KBMAX, int TR>
__device__ __forceinline__ void leaf_load_x(LeafSmem<T, KBMAX, TR> &sm, int kb, const T *__restrict__ X, int xs) {
    for (int idx = threadIdx.x; idx < kb * kb; idx += TR * 4) {
        const int i = idx / kb, l = idx - i * kb;
        sm.Ls[i][l] = l < i ? X[i * xs + l] : T(0);
    }
}

// Form (a): one CTA per tile, grid (row tiles, chunks).
template <typename T, int KBMAX>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 2)
leaf_update_kernel(T *W, long ld, int k, int kb, int coff, int N, int M, const T *__restrict__ X, int xs,
                   unsigned *tickets) {
    __shared__ LeafSmem<T, KBMAX, 64> sm;
    leaf_load_x(sm, kb, X, xs);
    leaf_tile<T, KBMAX, 64, false>(sm, W, ld, k, kb, coff, N, M, tickets, blockIdx.x * 64, blockIdx.y, gridDim.x,
                                   nullptr, nullptr);
}

// ---- left-looking U rows of the previous leaf over the trailing columns ----
// U_p = X_p (A12_p - L_p U_<p): A12_p = rows [kp, kp+kbp) of the columns
// [tc0, tc1) (after the leaf's row exchange), L_p = the same rows of the outer
// panel's columns [k0, kp), U_<p = rows [k0, kp) of the trailing columns (the
// U rows of the earlier leaves), X_p = the leaf's L11^{-1}.  One item is a
// chunk of kTrsmCols columns; the K = kp - k0 dimension streams through
// shared memory in tiles of kTrsmK rows, two tiles in flight (cp.async).
constexpr int kTrsmK = 32;

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(smem_dst)), "l"(gsrc),
                 "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <typename T, int KBMAX>
struct TrsmTile {
    static constexpr int CW = 512 / sizeof(T);  // columns per item (512-byte rows)
    __align__(16) T Lt[KBMAX][kTrsmK + 16 / sizeof(T)];
    __align__(16) T Ut[kTrsmK][CW];
};

template <typename T, int KBMAX>
__device__ void leaf_trsm_item(const LeafRestArgs<T> &p, int item, unsigned char *stage_raw) {
    using Tile = TrsmTile<T, KBMAX>;
    constexpr int CW = Tile::CW, NG = 512 / CW, RPTU = (KBMAX + NG - 1) / NG, VW = 16 / sizeof(T);
    static_assert(2 * sizeof(Tile) <= (size_t)kLeafStageBytes, "trsm tiles exceed the staging area");
    static_assert(sizeof(T) * KBMAX * CW + 4 * (512 / 32) <= 2 * sizeof(Tile), "U block and warp maxima exceed two tiles");
    static_assert((size_t)KBMAX * CW * sizeof(T) <= sizeof(Tile), "T block exceeds a tile");
    Tile *tl = reinterpret_cast<Tile *>(stage_raw);
    const int tid = threadIdx.x, c = tid % CW, g = tid / CW;
    const int cs = p.tc0 + item * CW, w = min(CW, p.tc1 - cs);
    const int K = p.kp - p.k0, nkt = (K + kTrsmK - 1) / kTrsmK;
    T *W = p.W;
    const long ld = p.ld;
    auto stage = [&](int t, Tile &b) {
        const int kk0 = t * kTrsmK;
        // L_p tile: kbp rows x kTrsmK columns of the outer panel
        constexpr int LV = kTrsmK / VW;
        for (int idx = tid; idx < p.kbp * LV; idx += 512) {
            const int r = idx / LV, q = idx - r * LV;
            const int kk = kk0 + q * VW;
            const int valid = max(0, min(VW, K - kk));
            // K is a multiple of VW: a piece is wholly inside or wholly outside
            const T *src = valid > 0 ? W + (long)(p.kp + r) * ld + p.k0 + kk : W;
            cp_async16(&b.Lt[r][q * VW], src, valid * (int)sizeof(T));
        }
        // U_<p tile: kTrsmK rows x CW columns
        constexpr int UV = CW / VW;
        for (int idx = tid; idx < kTrsmK * UV; idx += 512) {
            const int kr = idx / UV, q = idx - kr * UV;
            const int col = q * VW;
            const int valid = (kk0 + kr < K) ? max(0, min(VW, w - col)) : 0;
            const T *src = valid > 0 ? W + (long)(p.k0 + kk0 + kr) * ld + cs + col : W;
            cp_async16(&b.Ut[kr][col], src, valid * (int)sizeof(T));  // zero-filled past valid
        }
    };
    T acc[RPTU];
#pragma unroll
    for (int q = 0; q < RPTU; ++q) {
        const int r = g + NG * q;
        acc[q] = (r < p.kbp && c < w) ? W[(long)(p.kp + r) * ld + cs + c] : T(0);
    }
    if (nkt > 0) {
        stage(0, tl[0]);
        cp_async_commit();
    }
    for (int t = 0; t < nkt; ++t) {
        if (t + 1 < nkt) {
            stage(t + 1, tl[(t + 1) & 1]);
            cp_async_commit();
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const Tile &b = tl[t & 1];
#pragma unroll
        for (int k4 = 0; k4 < kTrsmK; k4 += VW) {
            T u[VW];
#pragma unroll
            for (int e = 0; e < VW; ++e) u[e] = b.Ut[k4 + e][c];
#pragma unroll
            for (int q = 0; q < RPTU; ++q) {
                const int r = g + NG * q;
                if (r < p.kbp) {  // warp-uniform
                    using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
                    const V lv = *reinterpret_cast<const V *>(&b.Lt[r][k4]);
                    const T *pl = reinterpret_cast<const T *>(&lv);
#pragma unroll
                    for (int e = 0; e < VW; ++e) acc[q] = fma(-pl[e], u[e], acc[q]);
                }
            }
        }
        __syncthreads();  // the buffer is refilled two tiles on
    }
    // U_p = X_p T (X_p unit lower), T through shared memory
    T(*Ts)[CW] = reinterpret_cast<T(*)[CW]>(stage_raw);
#pragma unroll
    for (int q = 0; q < RPTU; ++q) {
        const int r = g + NG * q;
        if (r < p.kbp) Ts[r][c] = acc[q];
    }
    __syncthreads();
    float vmax = 0.f;  // max |U| of this thread's values (NaN counted as infinite)
#pragma unroll
    for (int q = 0; q < RPTU; ++q) {
        const int r = g + NG * q;
        if (r < p.kbp && c < w) {
            T v = Ts[r][c];
            for (int l = 0; l < r; ++l) v = fma(p.Xp[r * p.xps + l], Ts[l][c], v);
            W[(long)(p.kp + r) * ld + cs + c] = v;
            const float a = fabsf((float)v);
            vmax = (a > vmax || a != a) ? ((a != a) ? INFINITY : a) : vmax;
        }
    }
    if (p.umax) {  // one atomic per item: warps, then the CTA
        float *wm = reinterpret_cast<float *>(stage_raw + sizeof(T) * KBMAX * CW);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, off));
        if ((tid & 31) == 0) wm[tid >> 5] = vmax;
        __syncthreads();
        if (tid == 0) {
            float m = 0.f;
            for (int i = 0; i < 512 / 32; ++i) m = fmaxf(m, wm[i]);
            atomicMax(p.umax, __float_as_uint(m));
        }
    }
    __syncthreads();  // Ts is reused by the next item
}

// Form (b): persistent, 128-row tiles; CTA b takes work items b, b +
// gridDim.x, ...: first the U rows of the previous leaf over the trailing
// columns (the longest items), then the update tiles (chunk-major, so
// consecutive CTAs share a chunk's A12 columns in L2), then the leaf's row
// exchange over the column ranges [0, mc1) and [mc2, mc3) (the columns
// outside the outer panel) in chunks of kMoveBytes, then the running row
// permutation perm.  An exchange item reads every source row of its chunk
// into shared memory before it writes any destination row, as the moves
// form cycles.  The previous leaf's rows are untouched by this leaf's moves
// (they act on rows >= k only), so its U items need no ordering against them.
constexpr int kMoveBytes = 512;

template <typename T, int KBMAX>
__global__ void __launch_bounds__(512, 1) leaf_update_persistent_kernel(const LeafRestArgs<T> p) {
    __shared__ LeafSmem<T, KBMAX, 128> sm;
    extern __shared__ __align__(16) unsigned char dyn_raw[];
    T *stage = reinterpret_cast<T *>(dyn_raw);
    unsigned *bits = reinterpret_cast<unsigned *>(dyn_raw + kLeafStageBytes);
    constexpr int CWm = kMoveBytes / sizeof(T);
    T *W = p.W;
    const long ld = p.ld;
    const int k = p.k, kb = p.kb, coff = p.coff, N = p.N, M = p.M, mc1 = p.mc1, mc2 = p.mc2, mc3 = p.mc3;
    const int2 *pairs = p.pairs;
    int *perm = p.perm;
    const int tid = threadIdx.x;
    const int NU = (p.kbp > 0 && p.tc1 > p.tc0) ? (p.tc1 - p.tc0 + TrsmTile<T, KBMAX>::CW - 1) / TrsmTile<T, KBMAX>::CW
                                                  : 0;
    const int R = max(1, (M + 127) / 128), C = (N > 0 && kb > 0) ? (N + kLeafTileCols - 1) / kLeafTileCols : 0;
    const int n1 = (mc1 + CWm - 1) / CWm, n2 = mc3 > mc2 ? (mc3 - mc2 + CWm - 1) / CWm : 0;
    const int np = p.npairs ? min(*p.npairs, 2 * KBMAX) : 0;
    const int nitems = NU + R * C + (np > 0 ? n1 + n2 : 0) + (perm && np > 0 ? 1 : 0);
    if ((int)blockIdx.x >= nitems) return;
    // the moves: A12 sources, the moved rows of A22 (list and bitmap)
    leaf_load_x(sm, kb, p.X, p.xs);
    if (tid < kb) sm.a12[tid] = k + tid;
    if (tid == 0) sm.nmv = 0;
    const int words = C > 0 ? (M + 31) / 32 : 0;
    for (int i = tid; i < words; i += blockDim.x) bits[i] = 0u;
    __syncthreads();
    for (int t = tid; t < np; t += blockDim.x) {
        const int2 mv = pairs[t];
        if (mv.x < k + kb) {
            sm.a12[mv.x - k] = mv.y;
        } else if (mv.x - (k + kb) < M && C > 0) {
            sm.mv[atomicAdd(&sm.nmv, 1)] = mv;
            const int rr = mv.x - (k + kb);
            atomicOr(&bits[rr >> 5], 1u << (rr & 31));
        }
    }
    __syncthreads();
    for (int t = blockIdx.x; t < nitems; t += gridDim.x) {
        if (t < NU) {
            leaf_trsm_item<T, KBMAX>(p, t, dyn_raw);
            continue;
        }
        const int t2 = t - NU;
        if (t2 < R * C) {
            const int chunk = t2 / R;
            leaf_tile<T, KBMAX, 128, true>(sm, W, ld, k, kb, coff, N, M, p.tickets, (t2 - chunk * R) * 128, chunk, R,
                                           bits, stage);
        } else if (t2 < R * C + n1 + n2) {
            const int q = t2 - R * C;
            const int cs = q < n1 ? q * CWm : mc2 + (q - n1) * CWm;
            const int ce = q < n1 ? min(cs + CWm, mc1) : min(cs + CWm, mc3);
            using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
            constexpr int VW = 16 / sizeof(T), NV = CWm / VW;
            V *tile = reinterpret_cast<V *>(stage);
            // cs is a multiple of CWm and ld of 32, so a vector is either
            // wholly inside [cs, ce) or (at the ragged end) read by elements
            for (int idx = tid; idx < np * NV; idx += blockDim.x) {
                const int pr = idx / NV, c = cs + (idx - pr * NV) * VW;
                const T *src = W + (long)pairs[pr].y * ld + c;
                if (c + VW <= ce) {
                    tile[idx] = *reinterpret_cast<const V *>(src);
                } else {
                    T *pv = reinterpret_cast<T *>(&tile[idx]);
                    for (int e = 0; e < VW; ++e) pv[e] = c + e < ce ? src[e] : T(0);
                }
            }
            __syncthreads();
            for (int idx = tid; idx < np * NV; idx += blockDim.x) {
                const int pr = idx / NV, c = cs + (idx - pr * NV) * VW;
                T *dst = W + (long)pairs[pr].x * ld + c;
                if (c + VW <= ce) {
                    *reinterpret_cast<V *>(dst) = tile[idx];
                } else {
                    const T *pv = reinterpret_cast<const T *>(&tile[idx]);
                    for (int e = 0; e < VW; ++e)
                        if (c + e < ce) dst[e] = pv[e];
                }
            }
        } else {  // the running row permutation
            int *pv = reinterpret_cast<int *>(stage);
            for (int i = tid; i < np; i += blockDim.x) pv[i] = perm[pairs[i].y];
            __syncthreads();
            for (int i = tid; i < np; i += blockDim.x) perm[pairs[i].x] = pv[i];
        }
        __syncthreads();  // the shared arrays are reused by the next item
    }
}

__global__ void apply_moves_vec_kernel(int *v, const int2 *pairs, const int *npairs) {
    extern __shared__ int vals[];
    const int np = *npairs;
    for (int t = threadIdx.x; t < np; t += blockDim.x) vals[t] = v[pairs[t].y];
    __syncthreads();
    for (int t = threadIdx.x; t < np; t += blockDim.x) v[pairs[t].x] = vals[t];
}

}  // namespace

cudaError_t launch_compose_swaps(const int32_t *ipiv, int k1, int k2, int n, int2 *pairs,
                                 int *npairs, int *map_scratch, cudaStream_t s) {
    const int npiv = k2 - k1, rows = n - k1;
    if (npiv <= 0) return cudaSuccess;
    size_t smem = sizeof(int) * (size_t)npiv;
    if (rows <= kComposeSmemRows) smem += sizeof(int) * (size_t)rows;
    cudaError_t e = mp_smem_attr(compose_swaps_kernel, smem);
    if (e != cudaSuccess) return e;
    mp_note_launch();
    compose_swaps_kernel<<<1, kComposeThreads, smem, s>>>(ipiv, k1, k2, n, pairs, npairs,
                                                          map_scratch);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_leaf_update(T *W, long ld, int k, int kb, int coff, int N, int M, const T *X, int xs,
                               unsigned *tickets, cudaStream_t s) {
    constexpr int KBMAX = sizeof(T) == 4 ? 24 : 8;
    if (N <= 0 || kb <= 0 || M < 0) return cudaSuccess;
    if (kb > KBMAX || N > 1024) return cudaErrorInvalidValue;
    dim3 grid(std::max(1, (M + 63) / 64), (N + kLeafTileCols - 1) / kLeafTileCols);
    mp_note_launch();
    leaf_update_kernel<T, KBMAX><<<grid, 256, 0, s>>>(W, ld, k, kb, coff, N, M, X, xs, tickets);
    return cudaGetLastError();
}
template cudaError_t launch_leaf_update<float>(float *, long, int, int, int, int, int, const float *, int,
                                              unsigned *, cudaStream_t);
template cudaError_t launch_leaf_update<double>(double *, long, int, int, int, int, int, const double *, int,
                                               unsigned *, cudaStream_t);

namespace {
template <typename T>
void leaf_rest_config(cudaLaunchConfig_t &cfg, cudaLaunchAttribute *attr, int clusters, int cluster,
                      cudaStream_t s) {
    cfg = cudaLaunchConfig_t{};
    cfg.gridDim = dim3(clusters * cluster, 1, 1);
    cfg.blockDim = dim3(512, 1, 1);
    cfg.dynamicSmemBytes = leaf_update_pad_bytes();
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
}
template <typename T>
cudaError_t leaf_rest_attrs() {
    constexpr int KBMAX = sizeof(T) == 4 ? 24 : 8;
    auto kern = leaf_update_persistent_kernel<T, KBMAX>;
    cudaError_t e = mp_smem_attr(kern, leaf_update_pad_bytes());
    if (e != cudaSuccess) return e;
    return mp_func_attr_once(reinterpret_cast<const void *>(kern), cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}
}  // namespace

template <typename T>
cudaError_t launch_leaf_rest(const LeafRestArgs<T> &p, int clusters, int cluster, cudaStream_t s) {
    constexpr int KBMAX = sizeof(T) == 4 ? 24 : 8;
    static_assert(2 * KBMAX * kMoveBytes <= kLeafStageBytes, "exchange tile exceeds the staging area");
    static_assert(2 * KBMAX * kLeafTileCols * (int)sizeof(T) <= kLeafStageBytes, "moved rows exceed the staging area");
    if (p.kb < 0 || p.M < 0 || p.N < 0 || clusters < 1 || cluster < 1 || cluster > 16) return cudaErrorInvalidValue;
    if (p.kb > KBMAX || p.N > 1024 || p.mc1 < 0 || p.mc3 < p.mc2 || p.M > kLeafMaxBitmapRows)
        return cudaErrorInvalidValue;
    if (p.kb > 0 && p.N > 0 && !p.X) return cudaErrorInvalidValue;
    if (p.kbp < 0 || p.kbp > KBMAX || (p.kbp > 0 && (!p.Xp || p.kp < p.k0 || (p.kp - p.k0) % (16 / (int)sizeof(T)))))
        return cudaErrorInvalidValue;
    cudaError_t e = leaf_rest_attrs<T>();
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    leaf_rest_config<T>(cfg, attr, clusters, cluster, s);
    mp_note_launch();
    return cudaLaunchKernelEx(&cfg, leaf_update_persistent_kernel<T, KBMAX>, p);
}
template cudaError_t launch_leaf_rest<float>(const LeafRestArgs<float> &, int, int, cudaStream_t);
template cudaError_t launch_leaf_rest<double>(const LeafRestArgs<double> &, int, int, cudaStream_t);

// Clusters of `cluster` CTAs of the persistent leaf update (one CTA per SM)
// that fit on the device at once, minus one: the remaining slot is left for
// the panel kernel of the same cluster size.  0 when no such split exists.
template <typename T>
int leaf_update_rest_clusters(int cluster) {
    static std::mutex mu;
    static int cache[2][64][17];
    static bool have[2][64][17];
    int dev = 0;
    if (cluster < 1 || cluster > 16 || cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    const int ti = sizeof(T) == 4 ? 0 : 1;
    std::lock_guard<std::mutex> g(mu);
    if (!have[ti][dev][cluster]) {
        constexpr int KBMAX = sizeof(T) == 4 ? 24 : 8;
        int nc = 0;
        if (leaf_rest_attrs<T>() == cudaSuccess) {
            cudaLaunchConfig_t cfg;
            cudaLaunchAttribute attr[1];
            leaf_rest_config<T>(cfg, attr, 1, cluster, nullptr);
            if (cudaOccupancyMaxActiveClusters(
                    &nc, reinterpret_cast<const void *>(leaf_update_persistent_kernel<T, KBMAX>), &cfg) != cudaSuccess)
                nc = 0;
        }
        cudaGetLastError();
        cache[ti][dev][cluster] = std::max(0, nc - 1);
        have[ti][dev][cluster] = true;
    }
    return cache[ti][dev][cluster];
}
template int leaf_update_rest_clusters<float>(int);
template int leaf_update_rest_clusters<double>(int);

template <typename T>
cudaError_t launch_apply_moves(T *W, long ld, const int2 *pairs, const int *npairs, int max_pairs,
                               int c0, int c1, int c2, int c3, int *perm, cudaStream_t s) {
    constexpr int CW = 128 / sizeof(T);  // 128-byte row segments
    if (c1 < c0) c1 = c0;
    if (c3 < c2) c3 = c2;
    int nch = (c1 - c0 + CW - 1) / CW + (c3 - c2 + CW - 1) / CW;
    if (max_pairs == 0) return cudaSuccess;
    if (nch == 0) {
        if (!perm) return cudaSuccess;
        nch = 1;  // perm only: one CTA whose column ranges are empty
    }
    size_t smem = (size_t)max_pairs * CW * sizeof(T);
    auto kern = apply_moves_kernel<T, CW>;
    cudaError_t e = mp_smem_attr(kern, smem);
    if (e != cudaSuccess) return e;
    mp_note_launch();
    kern<<<nch, 256, smem, s>>>(W, ld, pairs, npairs, c0, c1, c2, c3, perm);
    return cudaGetLastError();
}
template cudaError_t launch_apply_moves<float>(float *, long, const int2 *, const int *, int, int,
                                               int, int, int, int *, cudaStream_t);
template cudaError_t launch_apply_moves<double>(double *, long, const int2 *, const int *, int,
                                                int, int, int, int, int *, cudaStream_t);

cudaError_t launch_apply_moves_vec(int *v, const int2 *pairs, const int *npairs, int max_pairs,
                                   cudaStream_t s) {
    if (max_pairs == 0) return cudaSuccess;
    mp_note_launch();
    apply_moves_vec_kernel<<<1, 1024, sizeof(int) * (size_t)max_pairs, s>>>(v, pairs, npairs);
    return cudaGetLastError();
}

// ============================================================================
// C[MxN] -= A[MxK] B[KxN] with plain FMA in T (CUDA cores).  Used for the
// FP32 (and FP64 fallback) updates inside the panel and the triangular
// solve, and for the all-FP32 trailing update.
// 256 threads, BM x BN tile, BK-deep slices double-buffered through shared
// memory; each thread owns a TM x TN block split in two halves so that the
// shared-memory fragment reads are conflict free.
// ============================================================================
namespace {

// Batch addressing: entry z has offset (z / inner) * s_outer + (z % inner) * s_inner.
struct BatchStride {
    long s_outer, s_inner;
    __device__ __forceinline__ long off(int z, int inner) const {
        return (long)(z / inner) * s_outer + (long)(z % inner) * s_inner;
    }
};

// TB: B is given transposed (N x K row-major, C -= A B^T).  lower: skip the
// C tiles strictly above the diagonal (C square, symmetric update).
template <typename T, int BM, int BN, int BK, int TM, int TN, bool TB>
__global__ void __launch_bounds__(256)
gemm_kernel(int M, int N, int K, T alpha, T beta, const T *__restrict__ A0, long lda,
            const T *__restrict__ B0, long ldb, T *__restrict__ C0, long ldc, int inner,
            BatchStride sa, BatchStride sb, BatchStride sc, int lower) {
    static_assert((BM / TM) * (BN / TN) == 256, "thread layout");
    constexpr int TX = BN / TN;          // threads along N
    constexpr int A_ELEMS = BM * BK / 256;
    constexpr int B_ELEMS = BK * BN / 256;
    __shared__ T As[2][BK][BM];
    __shared__ T Bs[2][BK][BN];
    const int z = blockIdx.z;
    const T *A = A0 + sa.off(z, inner);
    const T *B = B0 + sb.off(z, inner);
    T *C = C0 + sc.off(z, inner);
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    if (lower && n0 > m0 + BM - 1) return;

    T ra[A_ELEMS], rb[B_ELEMS];
    auto load_tiles = [&](int k0) {
#pragma unroll
        for (int e = 0; e < A_ELEMS; ++e) {
            const int lin = tid * A_ELEMS + e;  // contiguous along k within a row
            const int r = lin / BK, kk = lin % BK;
            const int gr = m0 + r, gk = k0 + kk;
            ra[e] = (gr < M && gk < K) ? A[(long)gr * lda + gk] : T(0);
        }
#pragma unroll
        for (int e = 0; e < B_ELEMS; ++e) {
            const int lin = tid * B_ELEMS + e;  // contiguous along n (along k if TB)
            const int kk = TB ? lin % BK : lin / BN, c = TB ? lin / BK : lin % BN;
            const int gk = k0 + kk, gc = n0 + c;
            rb[e] = (gk < K && gc < N) ? (TB ? B[(long)gc * ldb + gk] : B[(long)gk * ldb + gc]) : T(0);
        }
    };
    auto store_tiles = [&](int buf) {
#pragma unroll
        for (int e = 0; e < A_ELEMS; ++e) {
            const int lin = tid * A_ELEMS + e;
            As[buf][lin % BK][lin / BK] = ra[e];
        }
#pragma unroll
        for (int e = 0; e < B_ELEMS; ++e) {
            const int lin = tid * B_ELEMS + e;
            if (TB) Bs[buf][lin % BK][lin / BK] = rb[e];
            else Bs[buf][lin / BN][lin % BN] = rb[e];
        }
    };

    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = T(0);

    const int KT = (K + BK - 1) / BK;
    if (KT > 0) {
        load_tiles(0);
        store_tiles(0);
    }
    __syncthreads();
    for (int kt = 0; kt < KT; ++kt) {
        const int cur = kt & 1;
        if (kt + 1 < KT) load_tiles((kt + 1) * BK);
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T af[TM], bf[TN];
#pragma unroll
            for (int i = 0; i < TM / 2; ++i) {
                af[i] = As[cur][kk][ty * (TM / 2) + i];
                af[i + TM / 2] = As[cur][kk][BM / 2 + ty * (TM / 2) + i];
            }
#pragma unroll
            for (int j = 0; j < TN / 2; ++j) {
                bf[j] = Bs[cur][kk][tx * (TN / 2) + j];
                bf[j + TN / 2] = Bs[cur][kk][BN / 2 + tx * (TN / 2) + j];
            }
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = fma(af[i], bf[j], acc[i][j]);
        }
        if (kt + 1 < KT) store_tiles(cur ^ 1);
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int r = m0 + (i < TM / 2 ? ty * (TM / 2) + i : BM / 2 + ty * (TM / 2) + (i - TM / 2));
        if (r >= M) continue;
        T *crow = C + (long)r * ldc;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int c = n0 + (j < TN / 2 ? tx * (TN / 2) + j : BN / 2 + tx * (TN / 2) + (j - TN / 2));
            if (c < N) crow[c] = (beta == T(0) ? T(0) : beta * crow[c]) + alpha * acc[i][j];
        }
    }
}

template <typename T>
cudaError_t gemm_launch(int M, int N, int K, T alpha, T beta, const T *A, long lda, const T *B, long ldb,
                        T *C, long ldc, int batch, int inner, BatchStride sa, BatchStride sb, BatchStride sc,
                        cudaStream_t s, bool tb = false, int lower = 0);

template <>
cudaError_t gemm_launch<float>(int M, int N, int K, float alpha, float beta, const float *A, long lda,
                               const float *B, long ldb, float *C, long ldc, int batch, int inner,
                               BatchStride sa, BatchStride sb, BatchStride sc, cudaStream_t s, bool tb,
                               int lower) {
    constexpr int BM = 128, BN = 128, BK = 8;
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, batch);
    mp_note_launch();
    if (tb)
        gemm_kernel<float, BM, BN, BK, 8, 8, true><<<grid, 256, 0, s>>>(M, N, K, alpha, beta, A, lda, B, ldb, C,
                                                                        ldc, inner, sa, sb, sc, lower);
    else
        gemm_kernel<float, BM, BN, BK, 8, 8, false><<<grid, 256, 0, s>>>(M, N, K, alpha, beta, A, lda, B, ldb, C,
                                                                         ldc, inner, sa, sb, sc, lower);
    return cudaGetLastError();
}
template <>
cudaError_t gemm_launch<double>(int M, int N, int K, double alpha, double beta, const double *A, long lda,
                                const double *B, long ldb, double *C, long ldc, int batch, int inner,
                                BatchStride sa, BatchStride sb, BatchStride sc, cudaStream_t s, bool tb,
                                int lower) {
    constexpr int BM = 64, BN = 64, BK = 16;
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, batch);
    mp_note_launch();
    if (tb)
        gemm_kernel<double, BM, BN, BK, 4, 4, true><<<grid, 256, 0, s>>>(M, N, K, alpha, beta, A, lda, B, ldb, C,
                                                                         ldc, inner, sa, sb, sc, lower);
    else
        gemm_kernel<double, BM, BN, BK, 4, 4, false><<<grid, 256, 0, s>>>(M, N, K, alpha, beta, A, lda, B, ldb, C,
                                                                          ldc, inner, sa, sb, sc, lower);
    return cudaGetLastError();
}

}  // namespace

template <typename T>
cudaError_t launch_gemm_sub(int M, int N, int K, const T *A, long lda, const T *B, long ldb, T *C, long ldc,
                            cudaStream_t s) {
    if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
    const BatchStride z{0, 0};
    return gemm_launch<T>(M, N, K, T(-1), T(1), A, lda, B, ldb, C, ldc, 1, 1, z, z, z, s);
}
template cudaError_t launch_gemm_sub<float>(int, int, int, const float *, long, const float *, long, float *,
                                            long, cudaStream_t);
template cudaError_t launch_gemm_sub<double>(int, int, int, const double *, long, const double *, long,
                                             double *, long, cudaStream_t);

template <typename T>
cudaError_t launch_gemm_nt_sub(int M, int N, int K, const T *A, long lda, const T *B, long ldb, T *C, long ldc,
                               int lower, cudaStream_t s) {
    if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
    const BatchStride z{0, 0};
    return gemm_launch<T>(M, N, K, T(-1), T(1), A, lda, B, ldb, C, ldc, 1, 1, z, z, z, s, true, lower);
}
template cudaError_t launch_gemm_nt_sub<float>(int, int, int, const float *, long, const float *, long, float *,
                                               long, int, cudaStream_t);
template cudaError_t launch_gemm_nt_sub<double>(int, int, int, const double *, long, const double *, long,
                                                double *, long, int, cudaStream_t);

template <typename T>
cudaError_t launch_gemm_batched(int M, int N, int K, T alpha, T beta, const T *A, long lda, const T *B, long ldb,
                                T *C, long ldc, int batch, int inner, long a_outer, long a_inner, long b_outer,
                                long b_inner, long c_outer, long c_inner, cudaStream_t s) {
    if (M <= 0 || N <= 0 || batch <= 0) return cudaSuccess;
    return gemm_launch<T>(M, N, K, alpha, beta, A, lda, B, ldb, C, ldc, batch, inner,
                          BatchStride{a_outer, a_inner}, BatchStride{b_outer, b_inner},
                          BatchStride{c_outer, c_inner}, s);
}
template cudaError_t launch_gemm_batched<float>(int, int, int, float, float, const float *, long, const float *,
                                                long, float *, long, int, int, long, long, long, long, long, long,
                                                cudaStream_t);
template cudaError_t launch_gemm_batched<double>(int, int, int, double, double, const double *, long,
                                                 const double *, long, double *, long, int, int, long, long, long,
                                                 long, long, long, cudaStream_t);

// ============================================================================
// B[m x N] <- L^{-1} B, L unit lower triangular (m <= 64).  One thread per
// column of B keeps the column in registers; L sits in shared memory.
// ============================================================================
namespace {

// B[m x N] <- L^{-1} B (m <= 64, L unit lower).  A CTA of 256 threads owns
// 64 columns of B; thread (q, c) holds rows 16q..16q+15 of column c.  Row
// blocks are finished in order: the owners of block q solve its 16 x 16
// diagonal triangle in registers and publish the values, then the owners of
// the later blocks subtract that block's contribution (16 independent
// accumulators per thread).  The published block is double-buffered: the
// writer of block q+1 cannot overwrite block q-1's values before every
// thread has passed the barrier after block q.
template <typename T>
__global__ void __launch_bounds__(256)
trsm_llnu_small_kernel(int m, int N, const T *__restrict__ L, long ldl, T *__restrict__ B, long ldb) {
    __shared__ T Ls[64][64];     // read as broadcasts (a warp shares q)
    __shared__ T Xs[2][16][64];  // the finished row block, double-buffered
    for (int idx = threadIdx.x; idx < 64 * 64; idx += blockDim.x) {
        const int i = idx / 64, l = idx % 64;
        Ls[i][l] = (i < m && l < i) ? L[(long)i * ldl + l] : T(0);
    }
    const int c = threadIdx.x & 63, q = threadIdx.x >> 6;
    const int col = blockIdx.x * 64 + c;
    const bool cv = col < N;
    T b[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int r = q * 16 + i;
        b[i] = (cv && r < m) ? B[(long)r * ldb + col] : T(0);
    }
    __syncthreads();
#pragma unroll 1
    for (int qb = 0; qb < 4; ++qb) {
        if (q == qb) {
#pragma unroll
            for (int i = 1; i < 16; ++i)
#pragma unroll
                for (int l = 0; l < i; ++l) b[i] = fma(-Ls[qb * 16 + i][qb * 16 + l], b[l], b[i]);
#pragma unroll
            for (int i = 0; i < 16; ++i) Xs[qb & 1][i][c] = b[i];
        }
        __syncthreads();
        if (q > qb) {
#pragma unroll
            for (int l = 0; l < 16; ++l) {
                const T x = Xs[qb & 1][l][c];
#pragma unroll
                for (int i = 0; i < 16; ++i) b[i] = fma(-Ls[q * 16 + i][qb * 16 + l], x, b[i]);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int r = q * 16 + i;
        if (cv && r < m) B[(long)r * ldb + col] = b[i];
    }
}

}  // namespace

template <typename T>
cudaError_t launch_trsm_llnu_small(int m, int N, const T *L, long ldl, T *B, long ldb, cudaStream_t s) {
    if (m <= 0 || N <= 0) return cudaSuccess;
    if (m > 64) return cudaErrorInvalidValue;
    mp_note_launch();
    trsm_llnu_small_kernel<T><<<(N + 63) / 64, 256, 0, s>>>(m, N, L, ldl, B, ldb);
    return cudaGetLastError();
}
template cudaError_t launch_trsm_llnu_small<float>(int, int, const float *, long, float *, long, cudaStream_t);
template cudaError_t launch_trsm_llnu_small<double>(int, int, const double *, long, double *, long, cudaStream_t);
