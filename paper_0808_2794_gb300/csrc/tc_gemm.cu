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
// E4M3 (kind::f8f6f4): every 128 x 128 block of L21 and of U12 has its own
// power-of-two scale (block max below 2^8); the kernel runs once per 128-wide
// K-block and the epilogue unscales each tile by its row block's and column
// block's scales of that K-block before subtracting it from C.
// Every mbarrier wait is bounded (about one second) and reports
// MP_FLAG_TIMEOUT instead of hanging.
#include <cuda.h>

#include <algorithm>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "common.cuh"
#include "tc_gemm.cuh"

namespace {

constexpr int TILE_J = 128;  // MMA M
constexpr int TILE_I = 256;  // MMA N
constexpr int BK = 64;       // 16-bit elements per 128-byte swizzled row
constexpr int A_BYTES = TILE_J * 128;  // one 128-byte row of K per operand row and stage
constexpr int B_BYTES = TILE_I * 128;
// FMT: 0 fp16, 1 bf16 (kind::f16, 64 K-elements per stage row), 2 E4M3
// (kind::f8f6f4, 128 K-elements per stage row); every MMA consumes 32 bytes
// of K.  E4M3 operands carry power-of-two scales (like the split rung).
template <uint32_t FMT> __host__ __device__ constexpr int bk_elems() { return FMT == 2 ? 128 : 64; }
template <uint32_t FMT, int SPLIT> __host__ __device__ constexpr bool scaled() { return SPLIT == 2 || FMT == 2; }
constexpr int NUM_EPI_WARPS = 8;
constexpr int NUM_THREADS = 64 + NUM_EPI_WARPS * 32;
constexpr uint32_t TMEM_COLS = 512;
constexpr int MAX_STAGES = 4;

// SPLIT = 1: one operand pair per stage (bf16 or fp16), 4 stages.
// SPLIT = 2: operands split in hi + lo fp16 parts (A_hi, A_lo, B_hi, B_lo per
//            stage), three products per k-step, 2 stages.
template <int SPLIT> struct TcCfg {
    static constexpr int STAGE_BYTES = SPLIT * (A_BYTES + B_BYTES);
    static constexpr int STAGES = SPLIT == 1 ? 4 : 2;
};

// Per-block scales of the E4M3 rung: the kernel handles K-block k_first
// (launched once per K-block), and tile (ib, jb) is unscaled by
// l_inv[rb * l_sr + k_first * l_sk] * u_inv[jb * u_sj + k_first * u_sk] with
// rb = its 128-row block (rows past the last block, nrb, are not stored).
// l_inv == nullptr: one scale for the whole product (*inv_scale_p).
struct BlockScales {
    const float *l_inv = nullptr, *u_inv = nullptr;
    int l_sr = 0, l_sk = 0, u_sj = 0, u_sk = 0, nrb = 0, k_first = 0;
};

struct __align__(8) TcBarriers {
    uint64_t full[MAX_STAGES];
    uint64_t empty[MAX_STAGES];
    uint64_t tfull[2];
    uint64_t tempty[2];
    uint32_t tmem_base;
    int abort_flag;
};

template <int SPLIT>
constexpr size_t smem_bytes() {
    return (size_t)TcCfg<SPLIT>::STAGES * TcCfg<SPLIT>::STAGE_BYTES + sizeof(TcBarriers) + 1024;
}

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
// Bounded wait: false after about one second (or limit_ns).
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, const volatile int *abort_flag,
                                          unsigned long long limit_ns = 1000000000ULL) {
    if (mbar_try_wait(a, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (long long i = 1;; ++i) {
        if (mbar_try_wait(a, parity)) return true;
        if ((i & 255) == 0) {
            if (*abort_flag) return false;
            if (global_ns() - t0 > limit_ns || i > (1LL << 32)) return false;
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
__device__ __forceinline__ void umma_f8(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
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

template <uint32_t FMT, int SPLIT>
__global__ void __launch_bounds__(NUM_THREADS, 1)
tc_update_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                 float *__restrict__ C, long ldc, int M, int N, int KB, int a_lo_row, int b_lo_row,
                 const float *__restrict__ inv_scale_p, MpDevStatus *st, int lower, BlockScales bs) {
    constexpr int STAGES = TcCfg<SPLIT>::STAGES;
    constexpr int STAGE_BYTES = TcCfg<SPLIT>::STAGE_BYTES;
    extern __shared__ unsigned char smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    TcBarriers *bar = reinterpret_cast<TcBarriers *>(smem + (size_t)STAGES * STAGE_BYTES);
    volatile int *abort_flag = &bar->abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int num_i = (M + TILE_I - 1) / TILE_I;
    const int num_j = (N + TILE_J - 1) / TILE_J;
    const int ntiles = num_i * num_j;
    // lower: tiles whose columns all lie right of their rows are skipped
    // (every role walks the same tile sequence, so the pipelines stay paired)
    auto skip = [&](int t) { return lower && (t / num_i) * TILE_J > (t % num_i) * TILE_I + TILE_I - 1; };

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
                if (skip(t)) continue;
                const int ib = t % num_i, jb = t / num_i;
                for (int kb = 0; kb < KB; ++kb) {
                    if (!mbar_wait(smem_u32(&bar->empty[stage]), phase ^ 1u, abort_flag)) { timed_out = true; break; }
                    const uint32_t sa = smem_u32(smem + (size_t)stage * STAGE_BYTES);
                    const uint32_t fb = smem_u32(&bar->full[stage]);
                    mbar_expect_tx(fb, STAGE_BYTES);
                    // stage layout: A_hi [A_lo] B_hi [B_lo]
                    constexpr int BKE = bk_elems<FMT>();
                    const int kx = (bs.k_first + kb) * BKE;
                    tma_load_2d(sa, &mapA, kx, jb * TILE_J, fb);
                    if (SPLIT == 2) tma_load_2d(sa + A_BYTES, &mapA, kx, a_lo_row + jb * TILE_J, fb);
                    tma_load_2d(sa + SPLIT * A_BYTES, &mapB, kx, ib * TILE_I, fb);
                    if (SPLIT == 2) tma_load_2d(sa + SPLIT * A_BYTES + B_BYTES, &mapB, kx, b_lo_row + ib * TILE_I, fb);
                    if (++stage == STAGES) { stage = 0; phase ^= 1u; }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {  // ---------------- MMA issuer
            constexpr uint32_t idesc = make_idesc(FMT == 2 ? 0u : FMT);  // E4M3 is format 0 of kind::f8f6f4
            int stage = 0;
            uint32_t phase = 0, acc_phase = 0;
            int acc = 0;
            for (int t = blockIdx.x; t < ntiles && !timed_out; t += gridDim.x) {
                if (skip(t)) continue;
                if (!mbar_wait(smem_u32(&bar->tempty[acc]), acc_phase ^ 1u, abort_flag)) { timed_out = true; break; }
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + (uint32_t)acc * TILE_I;
                for (int kb = 0; kb < KB; ++kb) {
                    if (!mbar_wait(smem_u32(&bar->full[stage]), phase, abort_flag)) { timed_out = true; break; }
                    tc_fence_after();
                    const uint32_t sa = smem_u32(smem + (size_t)stage * STAGE_BYTES);
                    const uint32_t sb = sa + SPLIT * A_BYTES;
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {  // 4 x 32 bytes of K per stage row
                        if constexpr (FMT == 2)
                            umma_f8(d_tmem, sw128_desc(sa + kk * 32), sw128_desc(sb + kk * 32), idesc,
                                    (kb | kk) ? 1u : 0u);
                        else
                            umma_f16(d_tmem, sw128_desc(sa + kk * 32), sw128_desc(sb + kk * 32), idesc,
                                     (kb | kk) ? 1u : 0u);
                        if (SPLIT == 2) {  // hi*lo and lo*hi
                            umma_f16(d_tmem, sw128_desc(sa + kk * 32), sw128_desc(sb + B_BYTES + kk * 32), idesc, 1u);
                            umma_f16(d_tmem, sw128_desc(sa + A_BYTES + kk * 32), sw128_desc(sb + kk * 32), idesc, 1u);
                        }
                    }
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
        const float inv_scale = scaled<FMT, SPLIT>() ? *inv_scale_p : 1.0f;
        int acc = 0;
        uint32_t acc_phase = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
            if (skip(t)) continue;
            const int ib = t % num_i, jb = t / num_i;
            if (!mbar_wait(smem_u32(&bar->tfull[acc]), acc_phase, abort_flag)) { timed_out = true; break; }
            tc_fence_after();
            const int col = jb * TILE_J + quarter * 32 + lane;
            const bool cval = col < N;
            // per-block scales (E4M3): this K-block's scale of the tile's 128-row
            // block of L21 times that of its 128-column block of U12
            float tinv = inv_scale;
            if (bs.l_inv) {
                const int rb = 2 * ib + half;
                tinv = rb < bs.nrb ? bs.l_inv[rb * bs.l_sr + bs.k_first * bs.l_sk] *
                                         bs.u_inv[jb * bs.u_sj + bs.k_first * bs.u_sk]
                                   : 0.f;
            }
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
                    if (cval && row0 + r < M) C[(long)(row0 + r) * ldc + col] = fmaf(-tinv, v[r], cv[r]);
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
// E4M3: round to nearest even, saturated to +-448 (OCP FP8)
template <> __device__ __forceinline__ __nv_fp8_e4m3 to_half<__nv_fp8_e4m3>(float v) { return __nv_fp8_e4m3(v); }

// Ap[j][k] = fl_p(U[k][j]) for j < N, k < Kpad (zero for k >= K): 32x32 transpose.
// SPLIT == 2: Ap[j] = fp16(s*u) (hi) and Ap[lo_row + j] = fp16(s*u - hi) (lo),
// s = *scale (a power of two).
template <typename H, int SPLIT>
__global__ void __launch_bounds__(256)
pack_transpose_kernel(int K, int N, int Kpad, const float *__restrict__ U, long ldu, H *__restrict__ Ap, long lo_row,
                      const float *__restrict__ scale, const float *__restrict__ bscale = nullptr, int bs_stride = 0) {
    __shared__ float t[32][33];
    const int j0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
    const float sc = (SPLIT == 2 || sizeof(H) == 1) ? *scale : 1.0f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int k = k0 + ty + 8 * q, j = j0 + tx;
        t[ty + 8 * q][tx] = (k < K && j < N) ? U[(long)k * ldu + j] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int j = j0 + ty + 8 * q, k = k0 + tx;
        if (j < N && k < Kpad) {
            // per-block scale of U's 128 x 128 block (k / 128, j / 128) when given
            const float v = t[tx][ty + 8 * q] * (bscale ? bscale[(k >> 7) * bs_stride + (j >> 7)] : sc);
            const H hi = to_half<H>(v);
            Ap[(long)j * Kpad + k] = hi;
            if constexpr (SPLIT == 2) Ap[(lo_row + j) * Kpad + k] = to_half<H>(v - __half2float(hi));
        }
    }
}

// Bp[i][k] = fl_p(L[i][k]) for i < M, k < Kpad (zero for k >= K); SPLIT as above.
// One warp per row (grid-stride over rows), lanes along k.
template <typename H, int SPLIT>
__global__ void __launch_bounds__(256)
pack_rows_kernel(int M, int K, int Kpad, const float *__restrict__ L, long ldl, H *__restrict__ Bp, long lo_row,
                 const float *__restrict__ scale, const float *__restrict__ bscale = nullptr, int bs_stride = 0) {
    const float sc = (SPLIT == 2 || sizeof(H) == 1) ? *scale : 1.0f;
    const int lane = threadIdx.x & 31;
    for (int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < M; i += gridDim.x * (blockDim.x >> 5)) {
        const float *src = L + (long)i * ldl;
        H *dst = Bp + (long)i * Kpad;
        const float *brow = bscale ? bscale + (long)(i >> 7) * bs_stride : nullptr;
        for (int k = lane; k < Kpad; k += 32) {
            // per-block scale of the 128 x 128 block (i / 128, k / 128) when given
            const float v = (k < K ? src[k] : 0.f) * (brow ? brow[k >> 7] : sc);
            const H hi = to_half<H>(v);
            dst[k] = hi;
            if constexpr (SPLIT == 2) dst[lo_row * Kpad + k] = to_half<H>(v - __half2float(hi));
        }
    }
}

// max |x| over a rows x cols row-major block -> *out (as uint bits of a non-negative float)
__global__ void __launch_bounds__(256)
absmax_kernel(int rows, int cols, const float *__restrict__ X, long ldx, unsigned *out) {
    float m = 0.f;
    // work items of one row x 1024 columns, one warp each (grid-stride)
    const int lane = threadIdx.x & 31;
    const int chunks = (cols + 1023) / 1024;
    const long items = (long)rows * chunks;
    for (long it = (long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); it < items;
         it += (long)gridDim.x * (blockDim.x >> 5)) {
        const int r = (int)(it / chunks), c0 = (int)(it - (long)r * chunks) * 1024;
        const float *xr = X + (long)r * ldx;
        const int c1 = min(cols, c0 + 1024);
#pragma unroll 8
        for (int c = c0 + lane; c < c1; c += 32) {
            const float v = fabsf(xr[c]);
            m = (v > m || v != v) ? ((v != v) ? INFINITY : v) : m;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

// Power-of-two scales: sU = 2^(top - ceil(log2 max|U|)) and sL = 2^(top - 1)
// when |l| <= 1 (partial pivoting), else sL from max|L| (lmax_bits) like
// sU; top = 14 for the split fp16 operands (below 65504), 8 for E4M3 (below
// 448); writes sL, sU and 1 / (sL sU).
__global__ void split_scales_kernel(const unsigned *umax_bits, const unsigned *lmax_bits, float *scales,
                                    int l_from_max, int top) {
    auto scale_exp = [top](unsigned bits) {
        const float m = __uint_as_float(bits);
        int e = 0;
        if (m > 0.f && m < INFINITY) frexpf(m, &e);  // m < 2^e
        return top - e;
    };
    const int eu = scale_exp(*umax_bits);
    const int el = l_from_max ? scale_exp(*lmax_bits) : top - 1;
    scales[0] = ldexpf(1.0f, el);
    scales[1] = ldexpf(1.0f, eu);
    scales[2] = ldexpf(1.0f, -el - eu);
}

// max |x| of every 128 x 128 block of a row-major rows x cols array into
// out[rb * ncb + cb] (bits of a non-negative float; NaN as +inf).  One CTA per
// block, consecutive threads along the block's rows (coalesced).
__global__ void __launch_bounds__(256)
block_absmax_kernel(int rows, int cols, const float *__restrict__ X, long ldx, unsigned *__restrict__ out, int ncb) {
    __shared__ float wm[8];
    const int r0 = blockIdx.y * 128, c0 = blockIdx.x * 128;
    float m = 0.f;
    for (int e = threadIdx.x; e < 128 * 128; e += 256) {
        const int r = r0 + (e >> 7), c = c0 + (e & 127);
        if (r < rows && c < cols) {
            const float v = fabsf(X[(long)r * ldx + c]);
            m = (v > m || v != v) ? ((v != v) ? INFINITY : v) : m;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = wm[0];
        for (int w = 1; w < 8; ++w) t = fmaxf(t, wm[w]);
        out[blockIdx.y * ncb + blockIdx.x] = __float_as_uint(t);
    }
}

// Per-block power-of-two scale 2^(top - e), max < 2^e (a zero or non-finite
// block: 2^top), and its inverse; the rule of split_scales_kernel per block.
__global__ void block_scales_kernel(int count, const unsigned *__restrict__ bits, float *__restrict__ scale,
                                    float *__restrict__ inv, int top) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const float m = __uint_as_float(bits[i]);
        int e = 0;
        if (m > 0.f && m < INFINITY) frexpf(m, &e);
        scale[i] = ldexpf(1.0f, top - e);
        inv[i] = ldexpf(1.0f, e - top);
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

// 2-D map over a (rows x kpad) K-major array of fmt (0 fp16, 1 bf16, 2 E4M3
// bytes), box (128 bytes of K x box_rows), 128B swizzle.
cudaError_t make_map(CUtensorMap *m, const void *base, long rows, int kpad, int box_rows, int fmt) {
    EncodeTiledFn enc = get_encode();
    if (!enc) return cudaErrorNotSupported;
    const int esz = fmt == 2 ? 1 : 2;
    cuuint64_t dims[2] = {(cuuint64_t)kpad, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)kpad * esz};
    cuuint32_t box[2] = {(cuuint32_t)(128 / esz), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    const CUtensorMapDataType dt = fmt == 2 ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                   : fmt == 1 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                              : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    CUresult r = enc(m, dt, 2,
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

struct TcWs {
    void *Ap, *Bp;
    unsigned *umax;
    float *scales;
    unsigned *lbits, *ubits;  // per-block maxima (E4M3)
    float *lsc, *linv, *usc, *uinv;
};

// Blocks of 128 x 128 of an operand with `rows` rows and K columns.
inline int blocks128(long v) { return (int)((v + 127) / 128); }

// Scratch layout: [Ap: rowsA x Kpad][Bp: rowsB x Kpad][umax, scales]
TcWs carve_ws(void *ws, int M, int N, int Kpad, int split, int esz) {
    const long rowsA = split == 2 ? 2L * ((N + TILE_J - 1) / TILE_J * TILE_J) : N;
    const long rowsB = split == 2 ? 2L * ((M + TILE_I - 1) / TILE_I * TILE_I) : M;
    char *p = static_cast<char *>(ws);
    TcWs w;
    w.Ap = p;
    p += align_up((size_t)rowsA * Kpad * esz, 1024);
    w.Bp = p;
    p += align_up((size_t)rowsB * Kpad * esz, 1024);
    w.umax = reinterpret_cast<unsigned *>(p);
    w.scales = reinterpret_cast<float *>(p + 16);
    p += 64;
    const size_t nbl = (size_t)blocks128(std::max(M, N)) * blocks128(Kpad);
    w.lbits = reinterpret_cast<unsigned *>(p);
    w.ubits = w.lbits + nbl;
    w.lsc = reinterpret_cast<float *>(w.ubits + nbl);
    w.linv = w.lsc + nbl;
    w.usc = w.linv + nbl;
    w.uinv = w.usc + nbl;
    return w;
}

// nt: U12 is given as its transpose (N x K row-major; C -= L21 U12t^T) and
// both split scales come from the operands' magnitudes.  lower: only the C
// tiles on or below the diagonal.
template <typename H, uint32_t FMT, int SPLIT>
cudaError_t run(int M, int N, int K, const float *L21, long ldl, const float *U12, long ldu, float *A22, long lda,
                void *ws, MpDevStatus *st, cudaStream_t s, bool nt = false, int lower = 0,
                const unsigned *umax_pre = nullptr) {
    constexpr int BKE = bk_elems<FMT>();
    constexpr bool SCALED = scaled<FMT, SPLIT>();
    const int Kpad = (K + BKE - 1) / BKE * BKE;
    TcWs w = carve_ws(ws, M, N, Kpad, SPLIT, (int)sizeof(H));
    const bool lmax = nt || FMT == 2;  // L's scale from its magnitude too
    H *Ap = reinterpret_cast<H *>(w.Ap);
    H *Bp = reinterpret_cast<H *>(w.Bp);
    const long a_lo = SPLIT == 2 ? (long)(N + TILE_J - 1) / TILE_J * TILE_J : 0;
    const long b_lo = SPLIT == 2 ? (long)(M + TILE_I - 1) / TILE_I * TILE_I : 0;
    cudaError_t e;
    const int KBk = Kpad / BKE;  // K-blocks (128 wide for E4M3)
    if (FMT == 2) {
        // per-128 x 128-block scales of L21 and U12 (E4M3)
        const int nrbL = blocks128(M), ncbU = blocks128(N);
        mp_note_launch(2);
        block_absmax_kernel<<<dim3(KBk, nrbL), 256, 0, s>>>(M, K, L21, ldl, w.lbits, KBk);
        if (nt)
            block_absmax_kernel<<<dim3(KBk, ncbU), 256, 0, s>>>(N, K, U12, ldu, w.ubits, KBk);
        else
            block_absmax_kernel<<<dim3(ncbU, KBk), 256, 0, s>>>(K, N, U12, ldu, w.ubits, ncbU);
        mp_note_launch(2);
        block_scales_kernel<<<(nrbL * KBk + 255) / 256, 256, 0, s>>>(nrbL * KBk, w.lbits, w.lsc, w.linv, 8);
        block_scales_kernel<<<(ncbU * KBk + 255) / 256, 256, 0, s>>>(ncbU * KBk, w.ubits, w.usc, w.uinv, 8);
    } else if (SCALED) {
        if (SPLIT == 2) {
            // the padding rows of both halves (up to the tile multiple) must be
            // zero; the pack kernels write every other element, K padding included
            auto zero_rows = [&](H *base, long r0, long r1) {
                return r1 > r0 ? cudaMemsetAsync(base + r0 * Kpad, 0, (size_t)(r1 - r0) * Kpad * sizeof(H), s)
                               : cudaSuccess;
            };
            if ((e = zero_rows(Ap, N, a_lo)) != cudaSuccess) return e;
            if ((e = zero_rows(Ap, a_lo + N, 2 * a_lo)) != cudaSuccess) return e;
            if ((e = zero_rows(Bp, M, b_lo)) != cudaSuccess) return e;
            if ((e = zero_rows(Bp, b_lo + M, 2 * b_lo)) != cudaSuccess) return e;
        }
        e = cudaMemsetAsync(w.umax, 0, 2 * sizeof(unsigned), s);
        if (e != cudaSuccess) return e;
        if (!umax_pre) {  // else max|U12| was taken while U12 was formed
            mp_note_launch();
            if (nt)
                absmax_kernel<<<1216, 256, 0, s>>>(N, K, U12, ldu, w.umax);
            else
                absmax_kernel<<<1216, 256, 0, s>>>(K, N, U12, ldu, w.umax);
        }
        if (lmax) {
            mp_note_launch();
            absmax_kernel<<<1216, 256, 0, s>>>(M, K, L21, ldl, w.umax + 1);
        }
        mp_note_launch();
        split_scales_kernel<<<1, 1, 0, s>>>(umax_pre ? umax_pre : w.umax, w.umax + 1, w.scales, lmax ? 1 : 0,
                                            FMT == 2 ? 8 : 14);
    }
    {
        const float *ubs = FMT == 2 ? w.usc : nullptr, *lbs = FMT == 2 ? w.lsc : nullptr;
        if (nt) {
            const long total = (long)N * Kpad;
            const int blocks = (int)std::min<long>((total + 255) / 256, 4L * 1024);
            mp_note_launch();
            pack_rows_kernel<H, SPLIT><<<blocks, 256, 0, s>>>(N, K, Kpad, U12, ldu, Ap, a_lo, w.scales + 1, ubs, KBk);
        } else {
            dim3 grid((N + 31) / 32, (Kpad + 31) / 32);
            mp_note_launch();
            pack_transpose_kernel<H, SPLIT><<<grid, 256, 0, s>>>(K, N, Kpad, U12, ldu, Ap, a_lo, w.scales + 1, ubs,
                                                                 blocks128(N));
        }
        const long total = (long)M * Kpad;
        const int blocks = (int)std::min<long>((total + 255) / 256, 4L * 1024);
        mp_note_launch();
        pack_rows_kernel<H, SPLIT><<<blocks, 256, 0, s>>>(M, K, Kpad, L21, ldl, Bp, b_lo, w.scales, lbs, KBk);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    CUtensorMap mapA, mapB;
    e = make_map(&mapA, Ap, SPLIT == 2 ? 2 * a_lo : N, Kpad, TILE_J, (int)FMT);
    if (e != cudaSuccess) return e;
    e = make_map(&mapB, Bp, SPLIT == 2 ? 2 * b_lo : M, Kpad, TILE_I, (int)FMT);
    if (e != cudaSuccess) return e;
    auto kern = tc_update_kernel<FMT, SPLIT>;
    constexpr size_t smem = smem_bytes<SPLIT>();
    e = mp_smem_attr(kern, smem);
    if (e != cudaSuccess) return e;
    const int ntiles = ((M + TILE_I - 1) / TILE_I) * ((N + TILE_J - 1) / TILE_J);
    const int grid = std::min(ntiles, num_sms());
    if (FMT == 2) {
        // one launch per K-block: each block's products carry their own scales
        BlockScales bs;
        bs.l_inv = w.linv;
        bs.l_sr = KBk;
        bs.l_sk = 1;
        bs.u_inv = w.uinv;
        bs.u_sj = nt ? KBk : 1;
        bs.u_sk = nt ? 1 : blocks128(N);
        bs.nrb = blocks128(M);
        for (int kb = 0; kb < KBk; ++kb) {
            bs.k_first = kb;
            mp_note_launch();
            kern<<<grid, NUM_THREADS, smem, s>>>(mapA, mapB, A22, lda, M, N, 1, (int)a_lo, (int)b_lo, w.scales + 2, st,
                                                 lower, bs);
        }
        return cudaGetLastError();
    }
    mp_note_launch();
    kern<<<grid, NUM_THREADS, smem, s>>>(mapA, mapB, A22, lda, M, N, KBk, (int)a_lo, (int)b_lo, w.scales + 2, st,
                                         lower, BlockScales{});
    return cudaGetLastError();
}

// Timeout path of the tensor-core kernels' bounded mbarrier wait, for the
// self-test: the barrier expects 16 bytes that nothing sends (site 4).
__global__ void selftest_tc_mbar_kernel(MpDevStatus *st, const int *abort_flag, unsigned long long limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&bar)), "r"(16u) : "memory");
    }
    __syncthreads();
    const bool ok = mbar_wait(smem_u32(&bar), 0u, abort_flag, limit_ns);
    if (!ok && threadIdx.x == 0) {
        mp_flag(st, MP_FLAG_TIMEOUT);
        atomicExch(&st->timeout_site, 4);
    }
}

}  // namespace

cudaError_t launch_selftest_tc_mbar(MpDevStatus *st, const int *abort_flag, unsigned long long limit_ns,
                                    cudaStream_t s) {
    mp_note_launch();
    selftest_tc_mbar_kernel<<<1, 32, 0, s>>>(st, abort_flag, limit_ns);
    return cudaGetLastError();
}

size_t tc_workspace_bytes(int n, int nb, int prec) {
    if (prec != MP_PREC_BF16 && prec != MP_PREC_FP16 && prec != MP_PREC_FP16X3 && prec != MP_PREC_E4M3) return 0;
    // 2-byte elements with K padded to 64 bound the E4M3 case (1 byte, K padded to 128)
    const size_t kpad = (size_t)(nb + BK - 1) / BK * BK;
    const int split = prec == MP_PREC_FP16X3 ? 2 : 1;
    const size_t rowsA = split == 2 ? 2 * ((size_t)(n + TILE_J - 1) / TILE_J * TILE_J) : (size_t)n;
    const size_t rowsB = split == 2 ? 2 * ((size_t)(n + TILE_I - 1) / TILE_I * TILE_I) : (size_t)n;
    // + the E4M3 per-block maxima, scales and inverses (6 arrays of 4 bytes per block)
    const size_t nbl = (size_t)((n + 127) / 128) * ((kpad + 127) / 128);
    return align_up(rowsA * kpad * 2, 1024) + align_up(rowsB * kpad * 2, 1024) + 1024 + 24 * nbl;
}

cudaError_t tc_trailing_update(int prec, int M, int N, int K, const float *L21, long ldl, const float *U12,
                               long ldu, float *A22, long lda, void *ws, MpDevStatus *st, cudaStream_t s,
                               const unsigned *umax_pre) {
    if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
    if (prec == MP_PREC_BF16)
        return run<__nv_bfloat16, 1, 1>(M, N, K, L21, ldl, U12, ldu, A22, lda, ws, st, s, false, 0, umax_pre);
    if (prec == MP_PREC_FP16)
        return run<__half, 0, 1>(M, N, K, L21, ldl, U12, ldu, A22, lda, ws, st, s, false, 0, umax_pre);
    if (prec == MP_PREC_FP16X3)
        return run<__half, 0, 2>(M, N, K, L21, ldl, U12, ldu, A22, lda, ws, st, s, false, 0, umax_pre);
    if (prec == MP_PREC_E4M3)
        return run<__nv_fp8_e4m3, 2, 1>(M, N, K, L21, ldl, U12, ldu, A22, lda, ws, st, s, false, 0, umax_pre);
    return cudaErrorInvalidValue;
}

cudaError_t tc_update_nt(int prec, int M, int N, int K, const float *A, long lda, const float *B, long ldb,
                         float *C, long ldc, int lower, void *ws, MpDevStatus *st, cudaStream_t s) {
    if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
    if (prec == MP_PREC_BF16) return run<__nv_bfloat16, 1, 1>(M, N, K, A, lda, B, ldb, C, ldc, ws, st, s, true, lower);
    if (prec == MP_PREC_FP16) return run<__half, 0, 1>(M, N, K, A, lda, B, ldb, C, ldc, ws, st, s, true, lower);
    if (prec == MP_PREC_FP16X3) return run<__half, 0, 2>(M, N, K, A, lda, B, ldb, C, ldc, ws, st, s, true, lower);
    if (prec == MP_PREC_E4M3)
        return run<__nv_fp8_e4m3, 2, 1>(M, N, K, A, lda, B, ldb, C, ldc, ws, st, s, true, lower);
    return cudaErrorInvalidValue;
}
