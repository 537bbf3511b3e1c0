// tc_gemm.cu -- the trailing-matrix update of the blocked LU on the
// Blackwell tensor cores: A22 <- A22 - fl_p(L21) fl_p(U12) (Section 2.1:
// the O(n^3) work, "the most computationally expensive operation", runs in
// the low precision; Section 3.1.1: the GEMM inside SGETRF).
//
// A22 is FP32 row-major (the working matrix W).  The kernel computes the
// transposed product D = U12^T L21^T so that a TMEM lane is a column of A22
// and the epilogue's global accesses are 128-byte coalesced rows:
//   MMA M (128) = columns j of A22     A operand: Ap[j][k] = fl_p(U12[k][j])
//   MMA N (256) = rows    i of A22     B operand: Bp[i][k] = fl_p(L21[i][k])
// Both operands are packed K-major (bf16/fp16, round to nearest even) and
// loaded by TMA with 128-byte swizzle into a 4-stage shared-memory ring.
// Warp roles (persistent CTA per SM): warp 0 = TMA producer, warp 1 = MMA
// issuer (tcgen05.mma.cta_group::1.kind::f16, FP32 accumulators in TMEM,
// two 256-column accumulators so the epilogue of tile t overlaps the MMAs of
// tile t+1), warps 2..9 = epilogue (tcgen05.ld, C - acc, coalesced stores).
// Every mbarrier wait is bounded (about one second) and reports
// MP_FLAG_TIMEOUT instead of hanging.
#include <cuda.h>

#include <algorithm>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "tc_gemm.cuh"

namespace {

constexpr int TILE_J = 128;  // MMA M
constexpr int TILE_I = 256;  // MMA N
constexpr int BK = 64;       // 16-bit elements per 128-byte swizzled row
constexpr int STAGES = 4;
constexpr int A_BYTES = TILE_J * BK * 2;
constexpr int B_BYTES = TILE_I * BK * 2;
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int NUM_EPI_WARPS = 8;
constexpr int NUM_THREADS = 64 + NUM_EPI_WARPS * 32;
constexpr uint32_t TMEM_COLS = 512;

struct __align__(8) TcBarriers {
    uint64_t full[STAGES];
    uint64_t empty[STAGES];
    uint64_t tfull[2];
    uint64_t tempty[2];
    uint32_t tmem_base;
    int abort_flag;
};

constexpr size_t kSmemBytes = (size_t)STAGES * STAGE_BYTES + sizeof(TcBarriers) + 1024;

// ---- PTX wrappers ------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t a) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t a, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: false after about one second.
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, const volatile int *abort_flag) {
    if (mbar_try_wait(a, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (long long i = 1;; ++i) {
        if (mbar_try_wait(a, parity)) return true;
        if ((i & 255) == 0) {
            if (*abort_flag) return false;
            if (global_ns() - t0 > 1000000000ULL || i > (1LL << 32)) return false;
        }
    }
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(mbar)
        : "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void tmem_ld_32x32b_x32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor: K-major operand tile, rows of 128 bytes,
// 128-byte swizzle, 8-row core groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;             // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset
    d |= (uint64_t)1 << 46;             // descriptor version
    d |= (uint64_t)2 << 61;             // SWIZZLE_128B
    return d;
}

// Instruction descriptor, kind::f16: D = F32, A/B = fmt (0 fp16, 1 bf16),
// both K-major, N = TILE_I, M = TILE_J.
__host__ __device__ constexpr uint32_t make_idesc(uint32_t fmt) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(TILE_I >> 3) << 17) |
           ((uint32_t)(TILE_J >> 4) << 24);
}

template <uint32_t FMT>
__global__ void __launch_bounds__(NUM_THREADS, 1)
tc_update_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                 float *__restrict__ C, long ldc, int M, int N, int KB, MpDevStatus *st) {
    extern __shared__ unsigned char smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    TcBarriers *bar = reinterpret_cast<TcBarriers *>(smem + (size_t)STAGES * STAGE_BYTES);
    volatile int *abort_flag = &bar->abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int num_i = (M + TILE_I - 1) / TILE_I;
    const int num_j = (N + TILE_J - 1) / TILE_J;
    const int ntiles = num_i * num_j;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(smem_u32(&bar->full[s]), 1);
            mbar_init(smem_u32(&bar->empty[s]), 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(smem_u32(&bar->tfull[a]), 1);
            mbar_init(smem_u32(&bar->tempty[a]), NUM_EPI_WARPS);
        }
        bar->abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapA)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapB)) : "memory");
    }
    if (warp == 1) {
        tmem_alloc(smem_u32(&bar->tmem_base), TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = bar->tmem_base;
    bool timed_out = false;

    if (warp == 0) {
        if (lane == 0) {  // ---------------- TMA producer
            int stage = 0;
            uint32_t phase = 0;
            for (int t = blockIdx.x; t < ntiles && !timed_out; t += gridDim.x) {
                const int ib = t % num_i, jb = t / num_i;
                for (int kb = 0; kb < KB; ++kb) {
                    if (!mbar_wait(smem_u32(&bar->empty[stage]), phase ^ 1u, abort_flag)) { timed_out = true; break; }
                    const uint32_t sa = smem_u32(smem + (size_t)stage * STAGE_BYTES);
                    const uint32_t fb = smem_u32(&bar->full[stage]);
                    mbar_expect_tx(fb, STAGE_BYTES);
                    tma_load_2d(sa, &mapA, kb * BK, jb * TILE_J, fb);
                    tma_load_2d(sa + A_BYTES, &mapB, kb * BK, ib * TILE_I, fb);
                    if (++stage == STAGES) { stage = 0; phase ^= 1u; }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {  // ---------------- MMA issuer
            constexpr uint32_t idesc = make_idesc(FMT);
            int stage = 0;
            uint32_t phase = 0, acc_phase = 0;
            int acc = 0;
            for (int t = blockIdx.x; t < ntiles && !timed_out; t += gridDim.x) {
                if (!mbar_wait(smem_u32(&bar->tempty[acc]), acc_phase ^ 1u, abort_flag)) { timed_out = true; break; }
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + (uint32_t)acc * TILE_I;
                for (int kb = 0; kb < KB; ++kb) {
                    if (!mbar_wait(smem_u32(&bar->full[stage]), phase, abort_flag)) { timed_out = true; break; }
                    tc_fence_after();
                    const uint32_t sa = smem_u32(smem + (size_t)stage * STAGE_BYTES);
                    const uint32_t sb = sa + A_BYTES;
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk)
                        umma_f16(d_tmem, sw128_desc(sa + kk * 32), sw128_desc(sb + kk * 32), idesc,
                                 (kb | kk) ? 1u : 0u);
                    umma_commit(smem_u32(&bar->empty[stage]));
                    if (++stage == STAGES) { stage = 0; phase ^= 1u; }
                }
                if (timed_out) break;
                umma_commit(smem_u32(&bar->tfull[acc]));
                acc ^= 1;
                if (acc == 0) acc_phase ^= 1u;
            }
        }
    } else {  // ------------------------------ epilogue warps 2..9
        const int quarter = warp & 3;        // TMEM lanes this warp may access
        const int half = (warp - 2) >> 2;    // which 128 of the 256 accumulator columns
        int acc = 0;
        uint32_t acc_phase = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
            const int ib = t % num_i, jb = t / num_i;
            if (!mbar_wait(smem_u32(&bar->tfull[acc]), acc_phase, abort_flag)) { timed_out = true; break; }
            tc_fence_after();
            const int col = jb * TILE_J + quarter * 32 + lane;
            const bool cval = col < N;
#pragma unroll 1
            for (int ch = 0; ch < 4; ++ch) {
                const int tcol = half * 128 + ch * 32;
                const int row0 = ib * TILE_I + tcol;
                float cv[32];
#pragma unroll
                for (int r = 0; r < 32; ++r)
                    cv[r] = (cval && row0 + r < M) ? C[(long)(row0 + r) * ldc + col] : 0.f;
                float v[32];
                tmem_ld_32x32b_x32(tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)acc * TILE_I + tcol, v);
#pragma unroll
                for (int r = 0; r < 32; ++r)
                    if (cval && row0 + r < M) C[(long)(row0 + r) * ldc + col] = cv[r] - v[r];
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&bar->tempty[acc]));
            acc ^= 1;
            if (acc == 0) acc_phase ^= 1u;
        }
    }
    if (timed_out) {
        *abort_flag = 1;
        mp_flag(st, MP_FLAG_TIMEOUT);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem_base, TMEM_COLS);
    }
}

// ---- operand packing ------------------------------------------------------------
template <typename H> __device__ __forceinline__ H to_half(float v);
template <> __device__ __forceinline__ __nv_bfloat16 to_half<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <> __device__ __forceinline__ __half to_half<__half>(float v) { return __float2half_rn(v); }

// Ap[j][k] = fl_p(U[k][j]) for j < N, k < Kpad (zero for k >= K): 32x32 transpose.
template <typename H>
__global__ void __launch_bounds__(256)
pack_transpose_kernel(int K, int N, int Kpad, const float *__restrict__ U, long ldu, H *__restrict__ Ap) {
    __shared__ float t[32][33];
    const int j0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int k = k0 + ty + 8 * q, j = j0 + tx;
        t[ty + 8 * q][tx] = (k < K && j < N) ? U[(long)k * ldu + j] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int j = j0 + ty + 8 * q, k = k0 + tx;
        if (j < N && k < Kpad) Ap[(long)j * Kpad + k] = to_half<H>(t[tx][ty + 8 * q]);
    }
}

// Bp[i][k] = fl_p(L[i][k]) for i < M, k < Kpad (zero for k >= K).
template <typename H>
__global__ void __launch_bounds__(256)
pack_rows_kernel(int M, int K, int Kpad, const float *__restrict__ L, long ldl, H *__restrict__ Bp) {
    const long total = (long)M * Kpad;
    for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
        const int i = (int)(idx / Kpad), k = (int)(idx - (long)i * Kpad);
        Bp[idx] = to_half<H>(k < K ? L[(long)i * ldl + k] : 0.f);
    }
}

// ---- host side -----------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// 2-D map over a (rows x kpad) K-major 16-bit array, box (64 x box_rows), 128B swizzle.
cudaError_t make_map(CUtensorMap *m, const void *base, int rows, int kpad, int box_rows, bool bf16) {
    EncodeTiledFn enc = get_encode();
    if (!enc) return cudaErrorNotSupported;
    cuuint64_t dims[2] = {(cuuint64_t)kpad, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)kpad * 2};
    cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
                     const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

int num_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 148;
    }
    return sms;
}

template <typename H, uint32_t FMT>
cudaError_t run(int M, int N, int K, const float *L21, long ldl, const float *U12, long ldu, float *A22,
                long lda, void *ws, MpDevStatus *st, cudaStream_t s) {
    const int Kpad = (K + BK - 1) / BK * BK;
    H *Ap = reinterpret_cast<H *>(ws);
    H *Bp = reinterpret_cast<H *>(static_cast<char *>(ws) + align_up((size_t)N * Kpad * sizeof(H), 1024));
    {
        dim3 grid((N + 31) / 32, (Kpad + 31) / 32);
        mp_note_launch();
        pack_transpose_kernel<H><<<grid, 256, 0, s>>>(K, N, Kpad, U12, ldu, Ap);
        const long total = (long)M * Kpad;
        const int blocks = (int)std::min<long>((total + 255) / 256, 4L * 1024);
        mp_note_launch();
        pack_rows_kernel<H><<<blocks, 256, 0, s>>>(M, K, Kpad, L21, ldl, Bp);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    CUtensorMap mapA, mapB;
    cudaError_t e = make_map(&mapA, Ap, N, Kpad, TILE_J, FMT == 1);
    if (e != cudaSuccess) return e;
    e = make_map(&mapB, Bp, M, Kpad, TILE_I, FMT == 1);
    if (e != cudaSuccess) return e;
    auto kern = tc_update_kernel<FMT>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    const int ntiles = ((M + TILE_I - 1) / TILE_I) * ((N + TILE_J - 1) / TILE_J);
    const int grid = std::min(ntiles, num_sms());
    mp_note_launch();
    kern<<<grid, NUM_THREADS, kSmemBytes, s>>>(mapA, mapB, A22, lda, M, N, Kpad / BK, st);
    return cudaGetLastError();
}

}  // namespace

size_t tc_workspace_bytes(int n, int nb, int prec) {
    if (prec != MP_PREC_BF16 && prec != MP_PREC_FP16) return 0;
    const size_t kpad = (size_t)(nb + BK - 1) / BK * BK;
    return align_up((size_t)n * kpad * 2, 1024) * 2 + 1024;
}

cudaError_t tc_trailing_update(int prec, int M, int N, int K, const float *L21, long ldl, const float *U12,
                               long ldu, float *A22, long lda, void *ws, MpDevStatus *st, cudaStream_t s) {
    if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
    if (prec == MP_PREC_BF16) return run<__nv_bfloat16, 1>(M, N, K, L21, ldl, U12, ldu, A22, lda, ws, st, s);
    if (prec == MP_PREC_FP16) return run<__half, 0>(M, N, K, L21, ldl, U12, ldu, A22, lda, ws, st, s);
    return cudaErrorInvalidValue;
}

cudaError_t tc_gemm_sub(int prec, int M, int N, int K, const float *A, long lda, const float *B, long ldb,
                        float *C, long ldc, void *ws, size_t ws_bytes, MpDevStatus *st, cudaStream_t s) {
    const int Kpad = (K + BK - 1) / BK * BK;
    const size_t need = align_up((size_t)N * Kpad * 2, 1024) + align_up((size_t)M * Kpad * 2, 1024);
    if (ws_bytes < need) return cudaErrorInvalidValue;
    return tc_trailing_update(prec, M, N, K, A, lda, B, ldb, C, ldc, ws, st, s);
}
