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
// U rows) go to shared memory.  Per column:
//   1. each thread finds its local candidate, warps reduce with shuffles
//      (largest magnitude, ties to the smallest row index, NaN counted as
//      infinite so it is chosen and reported as a breakdown); the winning
//      lane publishes its whole row in a per-warp slot, the owner of the
//      diagonal row publishes that row;                    -- CTA barrier
//   2. warp 0 reduces the warp candidates;                 -- cluster barrier
//   3. every warp reads the CTA candidates of the cluster and the winning and
//      diagonal rows through distributed shared memory, then rows are
//      exchanged, the column is scaled (true division) and the rank-1 update
//      is applied to the active columns.
// Slots are double-buffered, so two barriers per column suffice.  Every row
// carries the index of the row it came from; at the end the kernel writes
// the composed row permutation as (destination, source) moves for the row
// exchange of the rest of the matrix.
#include <climits>
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

template <typename T>
__device__ __forceinline__ Cand<T> warp_best(Cand<T> c) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const Cand<T> o = c.shfl_xor(off);
        if (o.better(c)) c = o;
    }
    return c;
}

template <typename T, int NB, int NT, int RPT>
struct PanelSmem {
    T fin[NT * RPT][NB + 1];        // finished values of the local rows (natural column order;
                                    // odd row stride: consecutive rows fall in different banks)
    T crow[2][NB];                  // this CTA's candidate row (double-buffered: read remotely)
    T drow[2][NB];                  // the diagonal row, if this CTA holds it
    __align__(16) T prow_s[2 * NB]; // pivot row in shifted coordinates: prow_s[t] = pivot[j + t]
    T prow[NB];                     // pivot row, natural columns
    T orow[NB];                     // old diagonal row, natural columns
    Cand<T> wkey[NT / 32];
    Cand<T> ckey[2];
    int corig[2];
    int dorig[2];
    int cidx, p, porig, dorg;
};

template <typename T, int NB, int RPT, int NT>
__global__ void __launch_bounds__(NT, 1)
panel_getf2_kernel(T *__restrict__ P, long ld, int m, int ncols, int row0, int32_t *__restrict__ ipiv,
                   int2 *__restrict__ moves, int *__restrict__ nmoves, MpDevStatus *st) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto &sm = *reinterpret_cast<PanelSmem<T, NB, NT, RPT> *>(smem_raw);
    using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
    constexpr int VW = 16 / sizeof(T);
    constexpr int NW = NT / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int CL = (int)cluster_nctarank();
    const int rank = (int)cluster_ctarank();
    const int rpc = (m + CL - 1) / CL;
    const int rbase = rank * rpc;
    if (rank == 0 && tid == 0) *nmoves = 0;
    for (int t = tid; t < 2 * NB; t += NT) sm.prow_s[t] = T(0);

    T a[RPT][NB];
    int gi[RPT], orig[RPT];
#pragma unroll
    for (int s = 0; s < RPT; ++s) {
        const int r = tid + s * NT;
        const int g = rbase + r;
        const bool valid = (r < rpc) && (g < m);
        gi[s] = valid ? g : INT_MAX;
        orig[s] = g;
        const T *row = P + (long)g * ld;
#pragma unroll
        for (int k = 0; k < NB; ++k) a[s][k] = (valid && k < ncols) ? row[k] : T(0);
    }

    int buf = 0;
#pragma unroll 1
    for (int j = 0; j < NB; ++j) {
        if (j < ncols) {  // uniform: dead steps only shift
            // ---- 1. warp candidates
            Cand<T> c = Cand<T>::none();
#pragma unroll
            for (int s = 0; s < RPT; ++s)
                if (gi[s] >= j && gi[s] < m) {
                    const Cand<T> o = Cand<T>::make(mag(a[s][0]), gi[s]);
                    if (o.better(c)) c = o;
                }
            c = warp_best(c);
            if (lane == 0) sm.wkey[warp] = c;
            __syncthreads();
            // ---- 2. the CTA candidate (warp 0)
            if (warp == 0) {
                Cand<T> cc = lane < NW ? sm.wkey[lane] : Cand<T>::none();
                cc = warp_best(cc);
                if (lane == 0) {
                    sm.ckey[buf] = cc;
                    sm.cidx = cc.idx();
                }
            }
            __syncthreads();
            // ---- 3. publish the CTA candidate row and the diagonal row (only the
            //         warps that hold them take the branch)
            const int ci = sm.cidx;
            bool mine_c = false, mine_d = false;
#pragma unroll
            for (int s = 0; s < RPT; ++s) {
                mine_c |= gi[s] == ci;
                mine_d |= gi[s] == j;
            }
            if (__any_sync(0xffffffffu, mine_c || mine_d)) {
#pragma unroll
                for (int s = 0; s < RPT; ++s) {
                    if (gi[s] == ci) {
                        const int lrow = tid + s * NT;
                        for (int k = 0; k < j; ++k) sm.crow[buf][k] = sm.fin[lrow][k];
#pragma unroll
                        for (int t = 0; t < NB; ++t)
                            if (j + t < NB) sm.crow[buf][j + t] = a[s][t];
                        sm.corig[buf] = orig[s];
                    }
                    if (gi[s] == j) {
                        const int lrow = tid + s * NT;
                        for (int k = 0; k < j; ++k) sm.drow[buf][k] = sm.fin[lrow][k];
#pragma unroll
                        for (int t = 0; t < NB; ++t)
                            if (j + t < NB) sm.drow[buf][j + t] = a[s][t];
                        sm.dorig[buf] = orig[s];
                    }
                }
            }
            if (CL > 1) cluster_sync_all(); else __syncthreads();
            // ---- 4. warp 0 reads the cluster's candidates and fetches the rows
            if (warp == 0) {
                Cand<T> g = Cand<T>::none();
                if (lane < CL) g = (CL > 1) ? Cand<T>::load_remote(mapa_shared(smem_u32(&sm.ckey[buf]), lane))
                                            : sm.ckey[buf];
                g = warp_best(g);
                const int p = g.idx();
                const int wr = p / rpc;  // CTA holding the pivot row
                const int dr = j / rpc;  // CTA holding the diagonal row
                // issue every remote load before using any of them
                T pv[(NB + 31) / 32], ov[(NB + 31) / 32];
                int po = 0, dor = 0;
#pragma unroll
                for (int q = 0; q < (NB + 31) / 32; ++q) {
                    const int k = lane + 32 * q;
                    if (k < NB) {
                        if (CL > 1) {
                            pv[q] = ld_dsmem<T>(mapa_shared(smem_u32(&sm.crow[buf][k]), wr));
                            ov[q] = ld_dsmem<T>(mapa_shared(smem_u32(&sm.drow[buf][k]), dr));
                        } else {
                            pv[q] = sm.crow[buf][k];
                            ov[q] = sm.drow[buf][k];
                        }
                    }
                }
                if (lane == 0) {
                    if (CL > 1) {
                        po = ld_dsmem_s32(mapa_shared(smem_u32(&sm.corig[buf]), wr));
                        dor = ld_dsmem_s32(mapa_shared(smem_u32(&sm.dorig[buf]), dr));
                    } else {
                        po = sm.corig[buf];
                        dor = sm.dorig[buf];
                    }
                }
#pragma unroll
                for (int q = 0; q < (NB + 31) / 32; ++q) {
                    const int k = lane + 32 * q;
                    if (k < NB) {
                        sm.prow[k] = pv[q];
                        sm.orow[k] = ov[q];
                        sm.prow_s[k - j + NB] = T(0);  // clear the tail left by earlier columns
                        if (k >= j) sm.prow_s[k - j] = pv[q];
                    }
                }
                if (lane == 0) {
                    sm.p = p;
                    sm.porig = po;
                    sm.dorg = dor;
                }
            }
            __syncthreads();
            const int p = sm.p;
            const T piv = sm.prow[j];
            if (rank == 0 && tid == 0) {
                ipiv[j] = row0 + p + 1;
                if (piv == T(0)) {
                    atomicCAS(&st->zero_pivot, 0, row0 + j + 1);
                    mp_flag(st, MP_FLAG_LOWP_BREAKDOWN);
                } else if (!(mag(piv) < T(INFINITY))) {
                    mp_flag(st, MP_FLAG_LOWP_BREAKDOWN);
                }
            }
            // ---- 5. row exchange (finished part in shared memory, active part in
            //         registers); only the warps holding row p or row j branch
            bool mine_x = false;
#pragma unroll
            for (int s = 0; s < RPT; ++s) mine_x |= (gi[s] == p && p != j) || gi[s] == j;
            if (__any_sync(0xffffffffu, mine_x)) {
#pragma unroll
                for (int s = 0; s < RPT; ++s) {
                    const bool is_p = gi[s] == p && p != j;
                    const bool is_j = gi[s] == j;
                    if (is_p || is_j) {
                        const T *src = is_p ? sm.orow : sm.prow;
                        const int lrow = tid + s * NT;
                        for (int k = 0; k < j; ++k) sm.fin[lrow][k] = src[k];
#pragma unroll
                        for (int t = 0; t < NB; ++t) a[s][t] = (j + t < NB) ? src[j + t] : T(0);
                        orig[s] = is_p ? sm.dorg : sm.porig;
                    }
                }
            }
            // ---- scale and rank-1 update of the active columns
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
            const V *pr4 = reinterpret_cast<const V *>(sm.prow_s);
#pragma unroll
            for (int q = 0; q < NB / VW; ++q) {
                const V v4 = pr4[q];
                const T *pv = reinterpret_cast<const T *>(&v4);
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
    __syncthreads();
    // write back the finished rows and the composed permutation
#pragma unroll
    for (int s = 0; s < RPT; ++s) {
        if (gi[s] < m) {
            T *row = P + (long)gi[s] * ld;
            const T *f = sm.fin[tid + s * NT];
            for (int k = 0; k < ncols; ++k) row[k] = f[k];
            if (orig[s] != gi[s]) {
                const int slot = atomicAdd(nmoves, 1);
                moves[slot] = make_int2(row0 + gi[s], row0 + orig[s]);
            }
        }
    }
    // no CTA may leave while a peer can still read its shared memory
    if (CL > 1) cluster_sync_all();
}

template <typename T, int NB, int RPT>
cudaError_t launch_panel_t(T *P, long ld, int m, int ncols, int row0, int32_t *ipiv, int2 *moves,
                           int *nmoves, MpDevStatus *st, cudaStream_t s) {
    constexpr int NT = 512;
    const int cap = NT * RPT;
    const int CL = (m + cap - 1) / cap;
    if (CL < 1 || CL > 16 || ncols > NB || ncols < 1 || m < ncols) return cudaErrorInvalidValue;
    auto kern = panel_getf2_kernel<T, NB, RPT, NT>;
    const size_t smem = sizeof(PanelSmem<T, NB, NT, RPT>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (CL > 8) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
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
    return cudaLaunchKernelEx(&cfg, kern, P, ld, m, ncols, row0, ipiv, moves, nmoves, st);
}

}  // namespace

// Base panel width for a panel of height m: one CTA keeps 1024 rows (float)
// of the panel in registers plus the finished part in shared memory, and a
// cluster has at most 16 CTAs.
template <>
int panel_base_width<float>(int m) {
    if (m <= 16384) return 32;
    if (m <= 32768) return 16;
    return 8;
}
template <>
int panel_base_width<double>(int m) {
    if (m <= 16384) return 16;
    if (m <= 32768) return 8;
    return 4;
}

template <>
cudaError_t launch_panel<float>(float *P, long ld, int m, int ncols, int row0, int32_t *ipiv, int2 *moves,
                                int *nmoves, MpDevStatus *st, cudaStream_t s) {
    if (m <= 16384) return launch_panel_t<float, 32, 2>(P, ld, m, ncols, row0, ipiv, moves, nmoves, st, s);
    if (m <= 32768) return launch_panel_t<float, 16, 4>(P, ld, m, ncols, row0, ipiv, moves, nmoves, st, s);
    return launch_panel_t<float, 8, 8>(P, ld, m, ncols, row0, ipiv, moves, nmoves, st, s);
}
template <>
cudaError_t launch_panel<double>(double *P, long ld, int m, int ncols, int row0, int32_t *ipiv, int2 *moves,
                                 int *nmoves, MpDevStatus *st, cudaStream_t s) {
    if (m <= 16384) return launch_panel_t<double, 16, 2>(P, ld, m, ncols, row0, ipiv, moves, nmoves, st, s);
    if (m <= 32768) return launch_panel_t<double, 8, 4>(P, ld, m, ncols, row0, ipiv, moves, nmoves, st, s);
    return launch_panel_t<double, 4, 8>(P, ld, m, ncols, row0, ipiv, moves, nmoves, st, s);
}
