// panel.cu -- pivoted LU of a tall, narrow panel (the unblocked kernel of
// the factorization PA = LU with partial row pivoting, Section 2.1;
// the LAPACK xGETF2 step inside SGETRF, Section 3.1.1).
//
// GB300 design: the panel (m rows x NB columns, row-major in W) is spread
// over a thread-block cluster of up to 16 CTAs and held entirely in
// registers (each thread owns RPT rows x NB columns).  Per column:
//   1. every CTA finds its local pivot candidate with warp-shuffle argmax
//      (largest magnitude, ties to the smallest row index; NaN counts as
//      infinite so that it is chosen and reported as a breakdown),
//   2. publishes (value, row, the whole candidate row) and the diagonal row
//      in its shared memory,
//   3. one cluster barrier,
//   4. every CTA reads the candidates of all CTAs through distributed
//      shared memory, picks the winner, exchanges rows in registers, scales
//      the column by the pivot (true division) and applies the rank-1 update
//      to the remaining columns.
// The published slots are double-buffered so one barrier per column suffices.
#include <climits>

#include "common.cuh"
#include "kernels.cuh"

namespace {

template <typename T, int NB, int NT>
struct PanelShared {
    T candrow[2][NB];
    T diagrow[2][NB];
    T pivrow[NB];
    T oldrow[NB];
    T candval[2];
    int candidx[2];
    T wv[NT / 32];
    int wi[NT / 32];
    int piv_idx;
};

template <typename T>
__device__ __forceinline__ T mag(T v) {
    T a = v < T(0) ? -v : v;
    return (a != a) ? T(INFINITY) : a;  // NaN -> +inf
}

template <typename T>
__device__ __forceinline__ void better(T &bv, int &bi, T ov, int oi) {
    if (ov > bv || (ov == bv && oi < bi)) {
        bv = ov;
        bi = oi;
    }
}

template <typename T, int NB, int RPT, int NT>
__global__ void __launch_bounds__(NT, 1)
panel_getf2_kernel(T *__restrict__ P, long ld, int m, int ncols, int row0,
                   int32_t *__restrict__ ipiv, MpDevStatus *st) {
    __shared__ PanelShared<T, NB, NT> sm;
    constexpr int NW = NT / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int CL = (int)cluster_nctarank();
    const int rank = (int)cluster_ctarank();
    const int rpc = (m + CL - 1) / CL;
    const int rbase = rank * rpc;

    T a[RPT][NB];
    int gi[RPT];
#pragma unroll
    for (int s = 0; s < RPT; ++s) {
        const int r = tid + s * NT;
        const int g = rbase + r;
        const bool valid = (r < rpc) && (g < m);
        gi[s] = valid ? g : INT_MAX;
        const T *row = P + (long)g * ld;
#pragma unroll
        for (int k = 0; k < NB; ++k) a[s][k] = (valid && k < ncols) ? row[k] : T(0);
    }

    int buf = 0;
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        if (j >= ncols) break;
        // ---- 1. local argmax over rows >= j
        T bv = T(-1);
        int bi = INT_MAX;
#pragma unroll
        for (int s = 0; s < RPT; ++s)
            if (gi[s] >= j && gi[s] < m) {
                const T v = mag(a[s][j]);
                if (v > bv) { bv = v; bi = gi[s]; }
            }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const T ov = __shfl_xor_sync(0xffffffffu, bv, off);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
            better(bv, bi, ov, oi);
        }
        if (lane == 0) { sm.wv[warp] = bv; sm.wi[warp] = bi; }
        __syncthreads();
        if (warp == 0) {
            bv = lane < NW ? sm.wv[lane] : T(-1);
            bi = lane < NW ? sm.wi[lane] : INT_MAX;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const T ov = __shfl_xor_sync(0xffffffffu, bv, off);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
                better(bv, bi, ov, oi);
            }
            if (lane == 0) { sm.candval[buf] = bv; sm.candidx[buf] = bi; }
        }
        __syncthreads();
        // ---- 2. publish the candidate row and the diagonal row
        const int cidx = sm.candidx[buf];
#pragma unroll
        for (int s = 0; s < RPT; ++s) {
            if (gi[s] == cidx) {
#pragma unroll
                for (int k = 0; k < NB; ++k) sm.candrow[buf][k] = a[s][k];
            }
            if (gi[s] == j) {
#pragma unroll
                for (int k = 0; k < NB; ++k) sm.diagrow[buf][k] = a[s][k];
            }
        }
        // ---- 3. exchange
        if (CL > 1) cluster_sync_all(); else __syncthreads();
        if (warp == 0) {
            T v = T(-1);
            int idx = INT_MAX;
            if (lane < CL) {
                if (CL > 1) {
                    v = ld_dsmem<T>(mapa_shared(smem_u32(&sm.candval[buf]), lane));
                    idx = ld_dsmem_s32(mapa_shared(smem_u32(&sm.candidx[buf]), lane));
                } else {
                    v = sm.candval[buf];
                    idx = sm.candidx[buf];
                }
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const T ov = __shfl_xor_sync(0xffffffffu, v, off);
                const int oi = __shfl_xor_sync(0xffffffffu, idx, off);
                better(v, idx, ov, oi);
            }
            const int wr = idx / rpc;  // CTA holding the pivot row
            const int dr = j / rpc;    // CTA holding the diagonal row
            for (int k = lane; k < NB; k += 32) {
                if (CL > 1) {
                    sm.pivrow[k] = ld_dsmem<T>(mapa_shared(smem_u32(&sm.candrow[buf][k]), wr));
                    sm.oldrow[k] = ld_dsmem<T>(mapa_shared(smem_u32(&sm.diagrow[buf][k]), dr));
                } else {
                    sm.pivrow[k] = sm.candrow[buf][k];
                    sm.oldrow[k] = sm.diagrow[buf][k];
                }
            }
            if (lane == 0) sm.piv_idx = idx;
        }
        __syncthreads();
        const int p = sm.piv_idx;
        const T piv = sm.pivrow[j];
        if (rank == 0 && tid == 0) {
            ipiv[j] = row0 + p + 1;
            if (piv == T(0)) {
                atomicCAS(&st->zero_pivot, 0, row0 + j + 1);
                mp_flag(st, MP_FLAG_LOWP_BREAKDOWN);
            } else if (!(mag(piv) < T(INFINITY))) {
                mp_flag(st, MP_FLAG_LOWP_BREAKDOWN);
            }
        }
        // ---- 4. row exchange, scaling, rank-1 update
#pragma unroll
        for (int s = 0; s < RPT; ++s) {
            if (gi[s] == p && p != j) {
#pragma unroll
                for (int k = 0; k < NB; ++k) a[s][k] = sm.oldrow[k];
            } else if (gi[s] == j) {
#pragma unroll
                for (int k = 0; k < NB; ++k) a[s][k] = sm.pivrow[k];
            }
        }
#pragma unroll
        for (int s = 0; s < RPT; ++s) {
            if (gi[s] > j && gi[s] < m) {
                T l = a[s][j];
                if (piv != T(0)) l = l / piv;
                a[s][j] = l;
#pragma unroll
                for (int k = j + 1; k < NB; ++k) a[s][k] = fma(-l, sm.pivrow[k], a[s][k]);
            }
        }
        buf ^= 1;
    }

#pragma unroll
    for (int s = 0; s < RPT; ++s) {
        if (gi[s] < m) {
            T *row = P + (long)gi[s] * ld;
#pragma unroll
            for (int k = 0; k < NB; ++k)
                if (k < ncols) row[k] = a[s][k];
        }
    }
    // no CTA may leave while a peer can still read its shared memory
    if (CL > 1) cluster_sync_all();
}

template <typename T, int NB, int RPT>
cudaError_t launch_panel_t(T *P, long ld, int m, int ncols, int row0, int32_t *ipiv,
                           MpDevStatus *st, cudaStream_t s) {
    constexpr int NT = 512;
    const int cap = NT * RPT;
    const int CL = (m + cap - 1) / cap;
    if (CL < 1 || CL > 16 || ncols > NB || ncols < 1 || m < ncols) return cudaErrorInvalidValue;
    auto kern = panel_getf2_kernel<T, NB, RPT, NT>;
    if (CL > 8) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL, 1, 1);
    cfg.blockDim = dim3(NT, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    mp_note_launch();
    return cudaLaunchKernelEx(&cfg, kern, P, ld, m, ncols, row0, ipiv, st);
}

}  // namespace

// Base panel width for a panel of height m: the register budget of one CTA
// is about 32K elements, and a cluster has at most 16 CTAs.
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
cudaError_t launch_panel<float>(float *P, long ld, int m, int ncols, int row0, int32_t *ipiv,
                                MpDevStatus *st, cudaStream_t s) {
    if (m <= 16384) return launch_panel_t<float, 32, 2>(P, ld, m, ncols, row0, ipiv, st, s);
    if (m <= 32768) return launch_panel_t<float, 16, 4>(P, ld, m, ncols, row0, ipiv, st, s);
    return launch_panel_t<float, 8, 8>(P, ld, m, ncols, row0, ipiv, st, s);
}
template <>
cudaError_t launch_panel<double>(double *P, long ld, int m, int ncols, int row0, int32_t *ipiv,
                                 MpDevStatus *st, cudaStream_t s) {
    if (m <= 16384) return launch_panel_t<double, 16, 2>(P, ld, m, ncols, row0, ipiv, st, s);
    if (m <= 32768) return launch_panel_t<double, 8, 4>(P, ld, m, ncols, row0, ipiv, st, s);
    return launch_panel_t<double, 4, 8>(P, ld, m, ncols, row0, ipiv, st, s);
}
