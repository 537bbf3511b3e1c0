// panel.cu -- pivoted LU of a tall, narrow panel (the unblocked kernel of
// the factorization PA = LU with partial row pivoting, Section 2.1;
// the LAPACK xGETF2 step inside SGETRF, Section 3.1.1).
//
// GB300 design.  The panel (m rows x NB columns, row-major in W) is spread
// over a thread-block cluster of up to 16 CTAs.  Each thread owns RPT rows.
// The columns that are still active live in registers and are shifted by one
// position after every column, so that the current column is always a[0] and
// the loop over columns is a rolled loop with static register indices (the
// body stays in the instruction cache).  Finished values (the L part and the
// U rows) go to shared memory.
//
// Prologue (optional, PanelPrev): the previous leaf of the same outer panel
// is applied to the panel's columns as they are loaded.  Rows are taken
// through that leaf's moves, U = X A12 is formed (X = its L11^{-1}), and
// A -= L21 U, so the panel is the only kernel on the critical path of a leaf.
//
// Per column:
//   1. each thread finds its local candidate and warps reduce with shuffles
//      (largest magnitude, ties to the smallest row index, NaN counted as
//      infinite so it is chosen and reported as a breakdown); the warp
//      candidates meet in shared memory                    -- CTA barrier
//   2. the warp holding the CTA's candidate row and the warp holding the
//      diagonal row push those rows into every CTA of the cluster
//      (st.async into distributed shared memory, counted on the receiver's
//      mbarrier; slots double-buffered by column)
//   3. every CTA waits on its mbarrier (bounded: a timeout sets a status flag
//      instead of hanging), picks the cluster's pivot, exchanges rows, scales
//      the column (true division) and applies the rank-1 update to the
//      active columns (paired FMAs; groups past the panel's edge skipped).
// Epilogue: X = L11^{-1} (warp-per-column substitution with shuffles), the
// previous leaf's U rows, the finished rows written back coalesced, and the
// composed row permutation as (destination, source) moves for the row
// exchange of the rest of the matrix.  Every row carries the index of the row
// it came from.
#include <algorithm>
#include <climits>
#include <cstddef>
#include <type_traits>

#include "common.cuh"
#include "kernels.cuh"

namespace {

template <typename T>
__device__ __forceinline__ T mag(T v) {
    T a = v < T(0) ? -v : v;
    return (a != a) ? T(INFINITY) : a;  // NaN -> +inf
}

// Pivot candidate: magnitude and row, ordered by magnitude, ties to the
// smaller row.  FP32 packs both into one 64-bit key (non-negative float bits
// order like unsigned integers), so a warp reduction is one 64-bit shuffle
// per round.  "No candidate" is the smallest key.
template <typename T> struct Cand;
template <> struct Cand<float> {
    unsigned long long k;
    __device__ __forceinline__ static Cand none() { return Cand{0ull}; }
    __device__ __forceinline__ static Cand make(float m, int idx) {
        return Cand{((unsigned long long)__float_as_uint(m) << 32) | (unsigned long long)(0xFFFFFFFFu - (unsigned)idx)};
    }
    __device__ __forceinline__ bool better(const Cand &o) const { return k > o.k; }
    __device__ __forceinline__ int idx() const { return k == 0ull ? INT_MAX : (int)(0xFFFFFFFFu - (unsigned)k); }
    __device__ __forceinline__ Cand shfl_xor(int off) const { return Cand{__shfl_xor_sync(0xffffffffu, k, off)}; }
    __device__ __forceinline__ static Cand load_remote(uint32_t addr) {
        unsigned long long v;
        asm volatile("ld.shared::cluster.u64 %0, [%1];" : "=l"(v) : "r"(addr) : "memory");
        return Cand{v};
    }
};
template <> struct Cand<double> {
    double v;
    int i;
    __device__ __forceinline__ static Cand none() { return Cand{-1.0, INT_MAX}; }
    __device__ __forceinline__ static Cand make(double m, int idx) { return Cand{m, idx}; }
    __device__ __forceinline__ bool better(const Cand &o) const { return v > o.v || (v == o.v && i < o.i); }
    __device__ __forceinline__ int idx() const { return i; }
    __device__ __forceinline__ Cand shfl_xor(int off) const {
        return Cand{__shfl_xor_sync(0xffffffffu, v, off), __shfl_xor_sync(0xffffffffu, i, off)};
    }
    __device__ __forceinline__ static Cand load_remote(uint32_t addr) {
        return Cand{ld_dsmem_f64(addr), ld_dsmem_s32(addr + 8)};
    }
};

// Warp-wide best candidate with redux.sync (maximum of the key words, most
// significant first); every lane receives it.
__device__ __forceinline__ Cand<float> warp_best(Cand<float> c) {
    const unsigned hi = (unsigned)(c.k >> 32), lo = (unsigned)c.k;
    const unsigned mhi = __reduce_max_sync(0xffffffffu, hi);
    const unsigned mlo = __reduce_max_sync(0xffffffffu, hi == mhi ? lo : 0u);
    return Cand<float>{((unsigned long long)mhi << 32) | mlo};
}
__device__ __forceinline__ Cand<double> warp_best(Cand<double> c) {
    // magnitude bits (non-negative doubles order like unsigned integers; "none"
    // maps to zero), then the smallest row among equal magnitudes
    const unsigned long long b = c.i == INT_MAX ? 0ull : (unsigned long long)__double_as_longlong(c.v);
    const unsigned inv = c.i == INT_MAX ? 0u : 0xFFFFFFFFu - (unsigned)c.i;
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const unsigned mhi = __reduce_max_sync(0xffffffffu, hi);
    const unsigned mlo = __reduce_max_sync(0xffffffffu, hi == mhi ? lo : 0u);
    const unsigned minv = __reduce_max_sync(0xffffffffu, (hi == mhi && lo == mlo) ? inv : 0u);
    if (minv == 0u) return Cand<double>::none();
    return Cand<double>{__longlong_as_double((long long)(((unsigned long long)mhi << 32) | mlo)),
                        (int)(0xFFFFFFFFu - minv)};
}

// Lane holding the best candidate among the lanes (the first such lane).
template <typename T>
__device__ __forceinline__ int best_lane(const Cand<T> &mine, const Cand<T> &best) {
    const bool eq = !(best.better(mine)) && !(mine.better(best));
    return __ffs(__ballot_sync(0xffffffffu, eq)) - 1;
}

// ---- push-based exchange inside a cluster ---------------------------------------
__device__ __forceinline__ void mbar_init_(uint32_t a, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arm(uint32_t a, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait (about one second, or limit_ns); false if it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t a, uint32_t parity,
                                                  unsigned long long limit_ns = 1000000000ULL) {
    for (int i = 0; i < 64; ++i)  // the usual case: the data arrives within a few polls
        if (mbar_try(a, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (long long i = 1;; ++i) {
        if (mbar_try(a, parity)) return true;
        if ((i & 255) == 0 && (global_ns() - t0 > limit_ns || i > (1LL << 30))) return false;
    }
}
// 16 bytes to the shared memory of another CTA of the cluster, counted on its mbarrier.
__device__ __forceinline__ void push16(uint32_t raddr, uint4 v, uint32_t rmbar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(raddr),
                 "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w), "r"(rmbar)
                 : "memory");
}

template <typename T, int NB>
struct __align__(16) Slot {  // one published row: key, origin, values (padded for shifted reads)
    Cand<T> key;
    int orig;
    alignas(16) T row[2 * NB];
};

template <typename T, int NB, int NT, int RPT>
struct PanelSmem {
    T fin[NT * RPT][NB + 1];   // finished values of the local rows (natural column order;
                               // odd row stride: consecutive rows fall in different banks)
    Slot<T, NB> rc[2][16];     // candidates received from every CTA (double-buffered by column)
    Slot<T, NB> rd[2];         // the diagonal row
    Slot<T, NB> stage[2];      // this CTA's outgoing candidate / diagonal row
    uint64_t mbar[2];
    Cand<T> wkey[2][NT / 32];  // per-warp candidates, double-buffered by column
    alignas(16) T wsh[NT / 32][NB];  // per-warp shifted pivot row
    // the previous leaf applied on load (PanelPrev; its width is at most NB)
    int redir[NT * RPT];          // local row -> row it takes its values from (INT_MIN: itself)
    int a12src[NB];               // previous leaf's row i -> its source row (relative to row0)
    int2 pp[2 * NB];              // its moves
    int np;
    T xp[NB][NB + 1];             // its X = L11^{-1}
    T ap[NB][NB];                 // A12 rows
    alignas(16) T up[NB][NB];     // U = X A12
};

// Columns [0, width) of rows rbase .. rbase+nvalid-1 of base (row-major, ld)
// into fin, coalesced: consecutive threads take consecutive 16-byte pieces of
// the rows (rows start on 16 bytes: ld and the column offsets are multiples of
// 4 floats / 2 doubles; checked at run time all the same).  BATCH loads are
// in flight at a time.
template <typename T, int NB, int NT, int RPT, int BATCH>
__device__ __forceinline__ void stage_rows(T (*fin)[NB + 1], const T *base, long ld, int rbase, int nvalid,
                                           int width) {
    using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
    constexpr int VW = 16 / sizeof(T), NV = NB / VW, ITEMS = RPT * NV;
    static_assert(ITEMS % BATCH == 0, "whole batches");
    const int tid = threadIdx.x;
    const bool vec = (reinterpret_cast<uintptr_t>(base) & 15) == 0;
#pragma unroll 1
    for (int it0 = 0; it0 < ITEMS; it0 += BATCH) {
        V buf[BATCH];
#pragma unroll
        for (int b = 0; b < BATCH; ++b) {
            const int idx = tid + (it0 + b) * NT, r = idx / NV, q = idx - r * NV;
            T *pv = reinterpret_cast<T *>(&buf[b]);
            if (r < nvalid && q * VW < width) {
                const T *src = base + (long)(rbase + r) * ld + q * VW;
                if (vec && (q + 1) * VW <= width) {
                    buf[b] = *reinterpret_cast<const V *>(src);
                } else {
#pragma unroll
                    for (int e = 0; e < VW; ++e) pv[e] = q * VW + e < width ? src[e] : T(0);
                }
            }
        }
#pragma unroll
        for (int b = 0; b < BATCH; ++b) {
            const int idx = tid + (it0 + b) * NT, r = idx / NV, q = idx - r * NV;
            const T *pv = reinterpret_cast<const T *>(&buf[b]);
            if (r < nvalid && q * VW < width) {
#pragma unroll
                for (int e = 0; e < VW; ++e) fin[r][q * VW + e] = pv[e];
            }
        }
    }
}

template <typename T, int NB, int RPT, int NT>
__global__ void __launch_bounds__(NT, 1)
panel_getf2_kernel(T *__restrict__ P, long ld, int m, int ncols, int row0, int32_t *__restrict__ ipiv,
                   int2 *__restrict__ moves, int *__restrict__ nmoves, MpDevStatus *st, T *__restrict__ linv,
                   PanelPrev<T> prev) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto &sm = *reinterpret_cast<PanelSmem<T, NB, NT, RPT> *>(smem_raw);
    constexpr int NW = NT / 32;
    using SlotT = Slot<T, NB>;
    constexpr int SLOT_HEAD = (int)offsetof(SlotT, row);  // bytes before the row values
    constexpr int ROW_BYTES = NB * (int)sizeof(T);
    static_assert(SLOT_HEAD % 16 == 0 && ROW_BYTES % 16 == 0, "16-byte pushes");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int CL = (int)cluster_nctarank();
    const int rank = (int)cluster_ctarank();
    const int rpc = (m + CL - 1) / CL;
    const int rbase = rank * rpc;
    const uint32_t bytes_per_col = (uint32_t)(CL + 1) * (SLOT_HEAD + ROW_BYTES);
    if (rank == 0 && tid == 0) *nmoves = 0;
    if (CL > 1) {
        if (tid == 0) {
            mbar_init_(smem_u32(&sm.mbar[0]), 1);
            mbar_init_(smem_u32(&sm.mbar[1]), 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            mbar_arm(smem_u32(&sm.mbar[0]), bytes_per_col);  // column 0
            mbar_arm(smem_u32(&sm.mbar[1]), bytes_per_col);  // column 1
        }
        cluster_sync_all();  // every mbarrier is armed before anyone pushes
    }

    T a[RPT][NB];
    int gi[RPT], orig[RPT];
    using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
    constexpr int VW = 16 / sizeof(T), NV = NB / VW;
    const int nvalid = max(0, min(rpc, m - rbase));  // rows of this CTA inside the panel
    // one row into registers
    auto load_row = [&](T (&dst)[NB], const T *row) {
        const bool vec_ok = (reinterpret_cast<uintptr_t>(row) & 15) == 0;
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            if (vec_ok && (q + 1) * VW <= ncols) {
                const V v = reinterpret_cast<const V *>(row)[q];
                const T *pv = reinterpret_cast<const T *>(&v);
#pragma unroll
                for (int e = 0; e < VW; ++e) dst[q * VW + e] = pv[e];
            } else {
#pragma unroll
                for (int e = 0; e < VW; ++e) {
                    const int k = q * VW + e;
                    dst[k] = k < ncols ? row[k] : T(0);
                }
            }
        }
    };
#pragma unroll
    for (int s = 0; s < RPT; ++s) {
        const int r = tid + s * NT;
        const int g = rbase + r;
        const bool valid = (r < rpc) && (g < m);
        gi[s] = valid ? g : INT_MAX;
        orig[s] = g;
        if (valid) {
            load_row(a[s], P + (long)g * ld);
        } else {
#pragma unroll
            for (int t = 0; t < NB; ++t) a[s][t] = T(0);
        }
    }

    // ---- 0. the previous leaf (PanelPrev): its moves, U = X A12 and
    //         A -= L21 U.  Rows are relative to row0; its rows are -kbp .. -1.
    //         First the moves, X and the L21 part of the local rows (staged
    //         in fin, which the column loop fills only later), then A12 and
    //         the rows the moves bring here.  Nothing is written to global
    //         memory before every CTA has finished reading: U and the panel's
    //         rows are stored after the column loop, whose first step waits
    //         for every CTA.
    const int kbp = prev.kb;
    if (kbp > 0) {
        if (tid < 2 * NB) sm.pp[tid] = prev.pairs[tid];  // slots past the count are never used
        if (tid == 0) sm.np = min(*prev.npairs, 2 * NB);
        for (int idx = tid; idx < kbp * kbp; idx += NT) {
            const int i = idx / kbp, l = idx - i * kbp;
            sm.xp[i][l] = prev.X[i * prev.xs + l];
        }
#pragma unroll
        for (int s = 0; s < RPT; ++s) sm.redir[tid + s * NT] = INT_MIN;
        // L21: the previous leaf's columns of the local rows (in batches: the
        // rows' values are live in registers meanwhile)
        stage_rows<T, NB, NT, RPT, NV>(sm.fin, P - kbp, ld, rbase, nvalid, kbp);
        if (tid < kbp) sm.a12src[tid] = tid - kbp;
        __syncthreads();
        for (int t = tid; t < sm.np; t += NT) {
            const int2 mv = sm.pp[t];
            const int d = mv.x - row0, src = mv.y - row0;
            if (d < 0) {
                if (d >= -kbp) sm.a12src[d + kbp] = src;
            } else if (d >= rbase && d < rbase + rpc) {
                sm.redir[d - rbase] = src;
            }
        }
        __syncthreads();
        for (int idx = tid; idx < kbp * NB; idx += NT) {
            const int i = idx / NB, c = idx - i * NB;
            sm.ap[i][c] = c < ncols ? P[(long)sm.a12src[i] * ld + c] : T(0);
        }
#pragma unroll
        for (int s = 0; s < RPT; ++s) {
            const int from = sm.redir[tid + s * NT];
            if (gi[s] < m && from != INT_MIN) load_row(a[s], P + (long)from * ld);
        }
        __syncthreads();
        // X unit lower: U row i = A12 row i + sum_{l<i} X_il A12 row l
        for (int idx = tid; idx < kbp * NB; idx += NT) {
            const int i = idx / NB, c = idx - i * NB;
            T v = sm.ap[i][c];
            for (int l = 0; l < i; ++l) v = fma(sm.xp[i][l], sm.ap[l][c], v);
            sm.up[i][c] = v;
        }
        __syncthreads();
        // A -= L21 U in the order l = 0 .. kbp-1 (each thread reads only its
        // own staged rows of fin, before the column loop writes them); row l
        // of U is read once for all of the thread's rows
        for (int l = 0; l < kbp; ++l) {
            T u[NB];
#pragma unroll
            for (int q = 0; q < NB / VW; ++q) {
                const V v = reinterpret_cast<const V *>(sm.up[l])[q];
                const T *pv = reinterpret_cast<const T *>(&v);
#pragma unroll
                for (int e = 0; e < VW; ++e) u[q * VW + e] = pv[e];
            }
#pragma unroll
            for (int s = 0; s < RPT; ++s) {
                const T lv = gi[s] < m ? sm.fin[tid + s * NT][l] : T(0);
                if constexpr (sizeof(T) == 4) {
#pragma unroll
                    for (int t = 0; t + 1 < NB; t += 2) {
                        const float2 r = fma2(make_float2(-lv, -lv), make_float2(u[t], u[t + 1]),
                                              make_float2(a[s][t], a[s][t + 1]));
                        a[s][t] = r.x;
                        a[s][t + 1] = r.y;
                    }
                } else {
#pragma unroll
                    for (int t = 0; t < NB; ++t) a[s][t] = fma(-lv, u[t], a[s][t]);
                }
            }
        }
    }

    bool ok = true;
    int buf = 0;
#pragma unroll 1
    for (int j = 0; j < NB; ++j) {
        if (j < ncols) {  // uniform: dead steps only shift
            // ---- 1. warp candidates -> CTA candidate (every warp reduces)
            Cand<T> c = Cand<T>::none();
#pragma unroll
            for (int s = 0; s < RPT; ++s)
                if (gi[s] >= j && gi[s] < m) {
                    const Cand<T> o = Cand<T>::make(mag(a[s][0]), gi[s]);
                    if (o.better(c)) c = o;
                }
            c = warp_best(c);
            // (a warp may already write column j + 1's key while a slower one
            // still reads column j's: the keys alternate between two buffers)
            if (lane == 0) sm.wkey[buf][warp] = c;
            __syncthreads();
            Cand<T> cc = lane < NW ? sm.wkey[buf][lane] : Cand<T>::none();
            cc = warp_best(cc);
            const int ci = cc.idx();
            const bool holds_diag = j >= rbase && j < rbase + rpc;
            // ---- 2. publish: the warp holding the CTA candidate (warp 0 if the CTA
            //         has none) and the warp holding the diagonal row stage their
            //         rows and push them to every CTA of the cluster
#pragma unroll
            for (int which = 0; which < 2; ++which) {
                int owner_row;
                if (which == 0) owner_row = ci;
                else {
                    if (!holds_diag) continue;
                    owner_row = j;
                }
                int owarp = 0, os = -1, olane = -1;
                if (owner_row != INT_MAX) {
                    const int lr = owner_row - rbase;
                    owarp = (lr % NT) / 32;
                    olane = (lr % NT) % 32;
                    os = lr / NT;
                }
                if (warp != owarp) continue;
                Slot<T, NB> &sg = sm.stage[which];
                if (os >= 0) {
                    const int lrow = warp * 32 + olane + os * NT;
                    for (int k = lane; k < j; k += 32) sg.row[k] = sm.fin[lrow][k];
                    if (lane == olane) {
#pragma unroll
                        for (int s = 0; s < RPT; ++s) {
                            if (s == os) {  // warp-uniform: os is the same in every lane
#pragma unroll
                                for (int t = 0; t < NB; ++t)
                                    if (j + t < NB) sg.row[j + t] = a[s][t];
                                sg.orig = orig[s];
                            }
                        }
                        sg.key = cc;
                    }
                } else if (lane == 0) {
                    sg.key = Cand<T>::none();
                    sg.orig = -1;
                }
                __syncwarp();
                // 16-byte chunks: head + row
                constexpr int CHUNKS = (SLOT_HEAD + ROW_BYTES) / 16;
                const uint4 *src = reinterpret_cast<const uint4 *>(&sg);
                if (CL > 1) {
                    for (int idx = lane; idx < CL * CHUNKS; idx += 32) {
                        const int dst = idx / CHUNKS, ch = idx - dst * CHUNKS;
                        const Slot<T, NB> *target = which == 0 ? &sm.rc[buf][rank] : &sm.rd[buf];
                        const uint32_t raddr = mapa_shared(smem_u32(target) + ch * 16, dst);
                        const uint32_t rmbar = mapa_shared(smem_u32(&sm.mbar[buf]), dst);
                        push16(raddr, src[ch], rmbar);
                    }
                } else {
                    uint4 *dstp = reinterpret_cast<uint4 *>(which == 0 ? &sm.rc[buf][0] : &sm.rd[buf]);
                    for (int ch = lane; ch < CHUNKS; ch += 32) dstp[ch] = src[ch];
                }
            }
            // ---- 3. wait for the candidates of every CTA and the diagonal row
            if (CL > 1) {
                if (!mbar_wait_bounded(smem_u32(&sm.mbar[buf]), (uint32_t)((j >> 1) & 1))) ok = false;
                __syncwarp();
            } else {
                __syncthreads();
            }
            const Cand<T> mine = lane < CL ? sm.rc[buf][lane].key : Cand<T>::none();
            const Cand<T> g = warp_best(mine);
            const int gw = best_lane(mine, g);
            const int p = g.idx();
            const Slot<T, NB> &ps = sm.rc[buf][gw];
            const Slot<T, NB> &ds = sm.rd[buf];
            const T piv = ps.row[j];
            if (rank == 0 && tid == 0) {
                ipiv[j] = row0 + p + 1;
                if (piv == T(0)) {
                    atomicCAS(&st->zero_pivot, 0, row0 + j + 1);
                    mp_flag(st, MP_FLAG_LOWP_BREAKDOWN);
                } else if (!(mag(piv) < T(INFINITY))) {
                    mp_flag(st, MP_FLAG_LOWP_BREAKDOWN);
                }
            }
            // ---- 4. row exchange; only the warps holding row p or row j branch.
            //         The finished part is copied by the whole warp.
            bool mine_x = false;
#pragma unroll
            for (int s = 0; s < RPT; ++s) mine_x |= (gi[s] == p && p != j) || gi[s] == j;
            const unsigned xmask = __ballot_sync(0xffffffffu, mine_x);
            if (xmask) {
                // at most two rows change; handle each owner lane in turn
                unsigned rem = xmask;
                while (rem) {
                    const int ol = __ffs(rem) - 1;
                    rem &= rem - 1;
#pragma unroll
                    for (int s = 0; s < RPT; ++s) {
                        const int g_s = __shfl_sync(0xffffffffu, gi[s], ol);
                        const bool is_p = g_s == p && p != j;
                        const bool is_j = g_s == j;
                        if (is_p || is_j) {  // warp-uniform
                            const T *src = is_p ? ds.row : ps.row;
                            const int lrow = warp * 32 + ol + s * NT;
                            for (int k = lane; k < j; k += 32) sm.fin[lrow][k] = src[k];
                            if (lane == ol) {
#pragma unroll
                                for (int t = 0; t < NB; ++t) a[s][t] = (j + t < NB) ? src[j + t] : T(0);
                                orig[s] = is_p ? ds.orig : ps.orig;
                            }
                        }
                    }
                }
            }
            // ---- 5. scale and rank-1 update of the active columns
            T l[RPT];
#pragma unroll
            for (int s = 0; s < RPT; ++s) {
                l[s] = T(0);
                if (gi[s] > j && gi[s] < m) {
                    l[s] = a[s][0];
                    if (piv != T(0)) l[s] = l[s] / piv;
                    a[s][0] = l[s];
                }
            }
            // the pivot row in shifted coordinates, 16-byte aligned, one copy per warp
            T *wsh = sm.wsh[warp];
            for (int t = lane; t < NB; t += 32) wsh[t] = (j + t < NB) ? ps.row[j + t] : T(0);
            __syncwarp();
            using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
            constexpr int VW = 16 / sizeof(T);
            const int act = ncols - j;  // a[.][t] with t < act are columns of the panel
#pragma unroll
            for (int q = 0; q < NB / VW; ++q) {
                if (q * VW >= act) continue;  // uniform: groups past the last column hold zeros
                const V v4 = reinterpret_cast<const V *>(wsh)[q];
                const T *pv = reinterpret_cast<const T *>(&v4);
                if constexpr (sizeof(T) == 4) {
                    // paired FMAs (fma.rn.f32x2, the same bits as two fmaf);
                    // t = 0 is column j itself, already scaled
#pragma unroll
                    for (int e = 0; e < VW; e += 2) {
                        const int t = q * VW + e;
#pragma unroll
                        for (int s = 0; s < RPT; ++s) {
                            if (t == 0) {
                                a[s][1] = fma(-l[s], pv[1], a[s][1]);
                            } else {
                                const float2 r = fma2(make_float2(-l[s], -l[s]), make_float2(pv[e], pv[e + 1]),
                                                      make_float2(a[s][t], a[s][t + 1]));
                                a[s][t] = r.x;
                                a[s][t + 1] = r.y;
                            }
                        }
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < VW; ++e) {
                        const int t = q * VW + e;
                        if (t >= 1) {
#pragma unroll
                            for (int s = 0; s < RPT; ++s) a[s][t] = fma(-l[s], pv[e], a[s][t]);
                        }
                    }
                }
            }
            // ---- 6. re-arm this buffer for column j + 2: no CTA can push that
            //         column before it has received our push of column j + 1,
            //         which comes after every thread here has left column j
            if (CL > 1 && tid == 0 && j + 2 < ncols) mbar_arm(smem_u32(&sm.mbar[buf]), bytes_per_col);
        }
        // ---- retire column j and shift the active columns
#pragma unroll
        for (int s = 0; s < RPT; ++s) {
            if (gi[s] < m) sm.fin[tid + s * NT][j] = a[s][0];
#pragma unroll
            for (int t = 0; t + 1 < NB; ++t) a[s][t] = a[s][t + 1];
            a[s][NB - 1] = T(0);
        }
        buf ^= 1;
    }
    if (!ok) mp_flag(st, MP_FLAG_TIMEOUT);
    __syncthreads();
    // X = L11^{-1} (unit lower, ncols x ncols; rows 0..ncols-1 are local rows
    // of CTA 0), row-major with stride NB.  Warp w forms the columns c = w,
    // w + NW, ... by column-oriented substitution: lane i holds x_i (x = e_c),
    // and for l = c, c+1, ... every lane i > l subtracts l_il x_l, x_l taken
    // from lane l.
    static_assert(NB <= 32, "one lane per row of L11");
    if (linv && rank == 0 && warp < ncols) {
        const int i = lane;
        T lrow[NB];
#pragma unroll
        for (int l = 0; l < NB; ++l) lrow[l] = (i < ncols && l < i) ? sm.fin[i][l] : T(0);
        for (int c = warp; c < ncols; c += NW) {
            T x = T(i == c ? 1 : 0);
#pragma unroll
            for (int l = 0; l < NB; ++l) {
                const T xl = __shfl_sync(0xffffffffu, x, l);
                if (l >= c && i > l) x = fma(-lrow[l], xl, x);
            }
            if (i < ncols) linv[i * NB + c] = x;
        }
    }
    // the previous leaf's U rows of these columns
    if (kbp > 0 && rank == 0)
        for (int idx = tid; idx < kbp * ncols; idx += NT) {
            const int i = idx / ncols, c = idx - i * ncols;
            P[(long)(i - kbp) * ld + c] = sm.up[i][c];
        }
    // write back the finished rows (coalesced, as stage_rows) and the
    // composed permutation
    {
        const bool vec = (reinterpret_cast<uintptr_t>(P) & 15) == 0;
#pragma unroll
        for (int it = 0; it < RPT * NV; ++it) {
            const int idx = tid + it * NT, r = idx / NV, q = idx - r * NV;
            if (r < nvalid && q * VW < ncols) {
                T *dst = P + (long)(rbase + r) * ld + q * VW;
                const T *src = &sm.fin[r][q * VW];
                if (vec && (q + 1) * VW <= ncols) {
                    V v;
                    T *pv = reinterpret_cast<T *>(&v);
#pragma unroll
                    for (int e = 0; e < VW; ++e) pv[e] = src[e];
                    *reinterpret_cast<V *>(dst) = v;
                } else {
#pragma unroll
                    for (int e = 0; e < VW; ++e)
                        if (q * VW + e < ncols) dst[e] = src[e];
                }
            }
        }
    }
#pragma unroll
    for (int s = 0; s < RPT; ++s)
        if (gi[s] < m && orig[s] != gi[s]) {
            const int slot = atomicAdd(nmoves, 1);
            moves[slot] = make_int2(row0 + gi[s], row0 + orig[s]);
        }
    // no CTA may leave while a peer can still push to it
    if (CL > 1) cluster_sync_all();
}

template <typename T, int NB, int RPT>
cudaError_t launch_panel_t(T *P, long ld, int m, int ncols, int row0, int32_t *ipiv, int2 *moves,
                           int *nmoves, MpDevStatus *st, T *linv, PanelPrev<T> prev, cudaStream_t s) {
    constexpr int NT = 512;
    const int cap = NT * RPT;
    const int CL = (m + cap - 1) / cap;
    if (CL < 1 || CL > 16 || ncols > NB || ncols < 1 || m < ncols) return cudaErrorInvalidValue;
    if (prev.kb < 0 || prev.kb > NB || (prev.kb > 0 && (!prev.X || !prev.pairs || !prev.npairs)))
        return cudaErrorInvalidValue;
    auto kern = panel_getf2_kernel<T, NB, RPT, NT>;
    const size_t smem = sizeof(PanelSmem<T, NB, NT, RPT>);
    cudaError_t e = mp_smem_attr(kern, smem);
    if (e != cudaSuccess) return e;
    if (CL > 8) {
        e = mp_func_attr_once(reinterpret_cast<const void *>(kern), cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL, 1, 1);
    cfg.blockDim = dim3(NT, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    mp_note_launch();
    return cudaLaunchKernelEx(&cfg, kern, P, ld, m, ncols, row0, ipiv, moves, nmoves, st, linv, prev);
}

// Timeout path of the panel's bounded mbarrier wait, for the self-test: the
// barrier expects 16 bytes that nothing sends (site 3).
__global__ void selftest_mbar_kernel(MpDevStatus *st, unsigned long long limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init_(smem_u32(&bar), 1);
        mbar_arm(smem_u32(&bar), 16);
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(smem_u32(&bar), 0u, limit_ns);
    if (!ok && threadIdx.x == 0) {
        mp_flag(st, MP_FLAG_TIMEOUT);
        atomicExch(&st->timeout_site, 3);
    }
}

}  // namespace

cudaError_t launch_selftest_panel_mbar(MpDevStatus *st, unsigned long long limit_ns, cudaStream_t s) {
    mp_note_launch();
    selftest_mbar_kernel<<<1, 32, 0, s>>>(st, limit_ns);
    return cudaGetLastError();
}

// Base panel width for a panel of height m.  One CTA keeps 1024 rows (512
// threads x 2 rows) of the active columns in registers and the finished part
// in shared memory; a cluster has at most 16 CTAs.  Widths are chosen so the
// register array stays well inside the 128-register budget of a 512-thread
// CTA (wider rows spill and cost more per column than they save in launches).
template <>
int panel_base_width<float>(int m) {
    if (m <= 16384) return 24;
    if (m <= 32768) return 16;
    return 8;
}
template <>
int panel_base_width<double>(int m) {
    if (m <= 16384) return 8;
    if (m <= 32768) return 8;
    return 4;
}

template <typename T>
int panel_cluster_size(int m) {
    const int rpt = m <= 16384 ? 2 : m <= 32768 ? 4 : 8;
    return std::max(1, (m + 512 * rpt - 1) / (512 * rpt));
}
template int panel_cluster_size<float>(int);
template int panel_cluster_size<double>(int);

template <>
cudaError_t launch_panel<float>(float *P, long ld, int m, int ncols, int row0, int32_t *ipiv, int2 *moves,
                                int *nmoves, MpDevStatus *st, float *linv, PanelPrev<float> prev,
                                cudaStream_t s) {
    if (m <= 16384) return launch_panel_t<float, 24, 2>(P, ld, m, ncols, row0, ipiv, moves, nmoves, st, linv, prev, s);
    if (m <= 32768) return launch_panel_t<float, 16, 4>(P, ld, m, ncols, row0, ipiv, moves, nmoves, st, linv, prev, s);
    return launch_panel_t<float, 8, 8>(P, ld, m, ncols, row0, ipiv, moves, nmoves, st, linv, prev, s);
}
template <>
cudaError_t launch_panel<double>(double *P, long ld, int m, int ncols, int row0, int32_t *ipiv, int2 *moves,
                                 int *nmoves, MpDevStatus *st, double *linv, PanelPrev<double> prev,
                                 cudaStream_t s) {
    if (m <= 16384) return launch_panel_t<double, 8, 2>(P, ld, m, ncols, row0, ipiv, moves, nmoves, st, linv, prev, s);
    if (m <= 32768) return launch_panel_t<double, 8, 4>(P, ld, m, ncols, row0, ipiv, moves, nmoves, st, linv, prev, s);
    return launch_panel_t<double, 4, 8>(P, ld, m, ncols, row0, ipiv, moves, nmoves, st, linv, prev, s);
}
