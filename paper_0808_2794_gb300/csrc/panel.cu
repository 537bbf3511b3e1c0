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

#include "common.cuh"
#include "kernels.cuh"

namespace {

template <typename T>
__device__ __forceinline__ T mag(T v) {
    T a = v < T(0) ? -v : v;
    return (a != a) ? T(INFINITY) : a;  // NaN -> +inf
}

template <typename T>
__device__ __forceinline__ void better(T &bv, int &bi, int &bw, T ov, int oi, int ow) {
    if (ov > bv || (ov == bv && oi < bi)) {
        bv = ov;
        bi = oi;
        bw = ow;
    }
}

template <typename T, int NB, int NT, int RPT>
struct PanelSmem {
    T fin[NT * RPT][NB];     // finished values of the local rows (natural column order)
    T wrow[2][NT / 32][NB];  // per-warp candidate rows
    T drow[2][NB];           // diagonal row
    T prow[NT / 32][2 * NB]; // per-warp copy of the pivot row (padded)
    T orow[NT / 32][NB];     // per-warp copy of the old diagonal row
    T wval[2][NT / 32];
    int widx[2][NT / 32];
    int worig[2][NT / 32];
    int dorig[2];
    T cval[2];
    int cidx[2];
    int cwarp[2];
};

template <typename T, int NB, int RPT, int NT>
__global__ void __launch_bounds__(NT, 1)
panel_getf2_kernel(T *__restrict__ P, long ld, int m, int ncols, int row0, int32_t *__restrict__ ipiv,
                   int2 *__restrict__ moves, int *__restrict__ nmoves, MpDevStatus *st) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto &sm = *reinterpret_cast<PanelSmem<T, NB, NT, RPT> *>(smem_raw);
    constexpr int NW = NT / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int CL = (int)cluster_nctarank();
    const int rank = (int)cluster_ctarank();
    const int rpc = (m + CL - 1) / CL;
    const int rbase = rank * rpc;
    if (rank == 0 && tid == 0) *nmoves = 0;

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
        const bool live = j < ncols;  // uniform: dead steps only shift
        int p = -1;
        if (live) {
            __syncwarp();  // retired values of the previous column are visible to the warp
            // ---- 1. candidates
            T bv = T(-1);
            int bi = INT_MAX, bo = -1, bs = -1;
#pragma unroll
            for (int s = 0; s < RPT; ++s)
                if (gi[s] >= j && gi[s] < m) {
                    const T v = mag(a[s][0]);
                    if (v > bv) { bv = v; bi = gi[s]; bo = orig[s]; bs = s; }
                }
            T wv = bv;
            int wi = bi, wl = lane;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const T ov = __shfl_xor_sync(0xffffffffu, wv, off);
                const int oi = __shfl_xor_sync(0xffffffffu, wi, off);
                const int ol = __shfl_xor_sync(0xffffffffu, wl, off);
                better(wv, wi, wl, ov, oi, ol);
            }
            // the winning lane publishes its row: finished part from shared
            // memory (copied by the whole warp), active part from registers
            const int ws_ = __shfl_sync(0xffffffffu, bs, wl);
            if (wi != INT_MAX) {
                const int lrow = (warp * 32 + wl) + ws_ * NT;
                for (int k = lane; k < j; k += 32) sm.wrow[buf][warp][k] = sm.fin[lrow][k];
                if (lane == wl) {
#pragma unroll
                    for (int s = 0; s < RPT; ++s)
                        if (s == bs) {
#pragma unroll
                            for (int t = 0; t < NB; ++t)
                                if (j + t < NB) sm.wrow[buf][warp][j + t] = a[s][t];
                        }
                    sm.wval[buf][warp] = bv;
                    sm.widx[buf][warp] = bi;
                    sm.worig[buf][warp] = bo;
                }
            } else if (lane == 0) {
                sm.wval[buf][warp] = T(-1);
                sm.widx[buf][warp] = INT_MAX;
            }
            // the diagonal row j
#pragma unroll
            for (int s = 0; s < RPT; ++s)
                if (gi[s] == j) {
                    const int lrow = tid + s * NT;
                    for (int k = 0; k < j; ++k) sm.drow[buf][k] = sm.fin[lrow][k];
#pragma unroll
                    for (int t = 0; t < NB; ++t)
                        if (j + t < NB) sm.drow[buf][j + t] = a[s][t];
                    sm.dorig[buf] = orig[s];
                }
            __syncthreads();
            // ---- 2. CTA candidate
            if (warp == 0) {
                T v = lane < NW ? sm.wval[buf][lane] : T(-1);
                int i = lane < NW ? sm.widx[buf][lane] : INT_MAX;
                int w = lane;
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    const T ov = __shfl_xor_sync(0xffffffffu, v, off);
                    const int oi = __shfl_xor_sync(0xffffffffu, i, off);
                    const int ow = __shfl_xor_sync(0xffffffffu, w, off);
                    better(v, i, w, ov, oi, ow);
                }
                if (lane == 0) { sm.cval[buf] = v; sm.cidx[buf] = i; sm.cwarp[buf] = w; }
            }
            if (CL > 1) cluster_sync_all(); else __syncthreads();
            // ---- 3. every warp reads the cluster's candidates
            T v = T(-1);
            int i = INT_MAX, w = 0, rk = lane;
            if (lane < CL) {
                if (CL > 1) {
                    v = ld_dsmem<T>(mapa_shared(smem_u32(&sm.cval[buf]), lane));
                    i = ld_dsmem_s32(mapa_shared(smem_u32(&sm.cidx[buf]), lane));
                    w = ld_dsmem_s32(mapa_shared(smem_u32(&sm.cwarp[buf]), lane));
                } else {
                    v = sm.cval[buf]; i = sm.cidx[buf]; w = sm.cwarp[buf];
                }
            }
            int wpack = w * 32 + rk;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const T ov = __shfl_xor_sync(0xffffffffu, v, off);
                const int oi = __shfl_xor_sync(0xffffffffu, i, off);
                const int ow = __shfl_xor_sync(0xffffffffu, wpack, off);
                better(v, i, wpack, ov, oi, ow);
            }
            p = i;
            const int wr = wpack & 31, ww = wpack >> 5;  // CTA and warp slot of the pivot row
            const int dr = j / rpc;                      // CTA holding the diagonal row
            int porig, dorig;
            if (CL > 1) {
                for (int k = lane; k < NB; k += 32) {
                    sm.prow[warp][k] = ld_dsmem<T>(mapa_shared(smem_u32(&sm.wrow[buf][ww][k]), wr));
                    sm.orow[warp][k] = ld_dsmem<T>(mapa_shared(smem_u32(&sm.drow[buf][k]), dr));
                }
                porig = ld_dsmem_s32(mapa_shared(smem_u32(&sm.worig[buf][ww]), wr));
                dorig = ld_dsmem_s32(mapa_shared(smem_u32(&sm.dorig[buf]), dr));
            } else {
                for (int k = lane; k < NB; k += 32) {
                    sm.prow[warp][k] = sm.wrow[buf][ww][k];
                    sm.orow[warp][k] = sm.drow[buf][k];
                }
                porig = sm.worig[buf][ww];
                dorig = sm.dorig[buf];
            }
            __syncwarp();
            const T piv = sm.prow[warp][j];
            if (rank == 0 && tid == 0) {
                ipiv[j] = row0 + p + 1;
                if (piv == T(0)) {
                    atomicCAS(&st->zero_pivot, 0, row0 + j + 1);
                    mp_flag(st, MP_FLAG_LOWP_BREAKDOWN);
                } else if (!(mag(piv) < T(INFINITY))) {
                    mp_flag(st, MP_FLAG_LOWP_BREAKDOWN);
                }
            }
            // ---- row exchange (finished part in shared memory, active part in registers)
#pragma unroll
            for (int s = 0; s < RPT; ++s) {
                const bool is_p = gi[s] == p && p != j;
                const bool is_j = gi[s] == j;
                if (is_p || is_j) {
                    const T *src = is_p ? sm.orow[warp] : sm.prow[warp];
                    const int lrow = tid + s * NT;
                    for (int k = 0; k < j; ++k) sm.fin[lrow][k] = src[k];
#pragma unroll
                    for (int t = 0; t < NB; ++t) a[s][t] = (j + t < NB) ? src[j + t] : T(0);
                    orig[s] = is_p ? dorig : porig;
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
            const T *prw = sm.prow[warp] + j;
#pragma unroll
            for (int t = 1; t < NB; ++t) {
                const T pv = prw[t];
#pragma unroll
                for (int s = 0; s < RPT; ++s) a[s][t] = fma(-l[s], pv, a[s][t]);
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
    __syncwarp();
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
