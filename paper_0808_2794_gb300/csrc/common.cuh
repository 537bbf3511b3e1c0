// common.cuh -- shared device/host helpers of the GB300 solver library.
//
// Layout convention inside the library: the low-precision working matrix W
// (FP32) and the FP64 fallback matrix are ROW-major (W[i*ld + j]).  Row
// exchanges of partial pivoting (Section 2.1) are then contiguous copies,
// the pivoted panel reads whole row segments, and the trailing update runs
// as the transposed product so that its epilogue stays coalesced.  The
// caller-facing matrices (A, B, X) are column-major.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mpsolve.h"

#define MP_CUDA_TRY(expr)                                   \
    do {                                                    \
        cudaError_t _e = (expr);                            \
        if (_e != cudaSuccess) return mp_cuda_fail(_e, #expr, __FILE__, __LINE__); \
    } while (0)

int mp_cuda_fail(cudaError_t e, const char *what, const char *file, int line);
int mp_arg_fail(int idx, const char *msg);
void mp_set_error(const char *msg);

// Device status block shared by the kernels of one solve.
struct MpDevStatus {
    uint32_t flags;        // MP_FLAG_* (atomicOr)
    int32_t zero_pivot;    // first zero pivot (1-based, atomicMin over positives) or 0
    int32_t timeout_site;  // where a bounded wait gave up (0 = none)
    int32_t pad;
    double anorm;          // ||A||_inf
};

__device__ __forceinline__ void mp_flag(MpDevStatus *st, uint32_t f) { atomicOr(&st->flags, f); }

// Non-negative doubles order like their bit patterns: max via 64-bit atomicMax.
__device__ __forceinline__ void atomic_max_nonneg(double *addr, double v) {
    if (!(v >= 0.0)) v = __longlong_as_double(0x7ff0000000000000LL);  // NaN -> +inf
    atomicMax(reinterpret_cast<unsigned long long *>(addr),
              static_cast<unsigned long long>(__double_as_longlong(v)));
}

// ---- thread-block cluster helpers (inline PTX, sm_90+) ---------------------
// Two FP32 FMAs in one instruction (the paired FMA of sm_100 and later,
// element-wise, round to nearest even): d = a * b + c lane by lane, the same
// bits as two fmaf calls.  The builtin lets the register allocator keep the
// operands in register pairs.
// fl32(v): v rounded to binary32, to nearest with ties to even, computed
// from the IEEE 754 binary64 and binary32 encodings with 32-bit integer
// operations only.  GB300's FP64 pipe issues a small fraction of the integer
// rate, so an n^2 conversion that converts with the FP64 unit is bound by it
// rather than by HBM.  Normal results take the first branch: keep 23 of the 52
// fraction bits, round on the 29 dropped ones (a carry out of the fraction
// raises the exponent, and from the largest exponent gives infinity).
static __device__ __noinline__ uint32_t fl32_bits_rare(uint32_t hi, uint32_t lo) {
    const uint32_t sign = hi & 0x80000000u;
    const int ex = (int)((hi >> 20) & 0x7ffu);
    const uint32_t frac_hi = hi & 0xfffffu;
    if (ex == 0x7ff)  // infinity, or NaN (quiet, keeping the top payload bits)
        return (frac_hi | lo) ? (sign | 0x7fc00000u | (frac_hi << 3) | (lo >> 29)) : (sign | 0x7f800000u);
    if (ex >= 1151) return sign | 0x7f800000u;  // |v| >= 2^128: beyond the largest binary32 after rounding
    // binary32 subnormal or zero: the significand in units of 2^-149
    const unsigned long long M = ((unsigned long long)(ex ? (frac_hi | 0x100000u) : frac_hi) << 32) | lo;
    const int sh = ex ? 926 - ex : 925;  // >= 30 here
    if (sh > 63) return sign;  // |v| < 2^-150: rounds to zero
    unsigned long long q = M >> sh;
    const unsigned long long rem = M & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    q += (rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull;
    return sign | (uint32_t)q;  // 2^23 after rounding is the smallest normal
}

__device__ __forceinline__ float fl32_rne(double v) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(v);
    const uint32_t hi = (uint32_t)(u >> 32), lo = (uint32_t)u;
    const uint32_t fe = ((hi >> 20) & 0x7ffu) - 896u;  // binary32 biased exponent (wraps when below 1)
    if (fe - 1u < 254u) {
        uint32_t f = (fe << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
        const uint32_t r = lo & 0x1fffffffu;
        f += (r > 0x10000000u || (r == 0x10000000u && (f & 1u))) ? 1u : 0u;
        return __uint_as_float((hi & 0x80000000u) | f);
    }
    return __uint_as_float(fl32_bits_rare(hi, lo));
}

// v is infinite or NaN (exponent field all ones), tested on the high word
__device__ __forceinline__ bool nonfinite_f64(double v) {
    return ((uint32_t)__double2hiint(v) & 0x7ff00000u) == 0x7ff00000u;
}

__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

__device__ __forceinline__ uint32_t cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_nctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Map a local shared-memory address to the same variable in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint32_t mapa_shared(uint32_t addr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}
__device__ __forceinline__ float ld_dsmem_f32(uint32_t addr) {
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(addr) : "memory");
    return v;
}
__device__ __forceinline__ double ld_dsmem_f64(uint32_t addr) {
    double v;
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(addr) : "memory");
    return v;
}
__device__ __forceinline__ int ld_dsmem_s32(uint32_t addr) {
    int v;
    asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}
template <typename T> __device__ __forceinline__ T ld_dsmem(uint32_t addr);
template <> __device__ __forceinline__ float ld_dsmem<float>(uint32_t a) { return ld_dsmem_f32(a); }
template <> __device__ __forceinline__ double ld_dsmem<double>(uint32_t a) { return ld_dsmem_f64(a); }

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---- grid-wide barrier for a cooperative launch (bounded wait: after
//      limit_ns without the last arrival a CTA records a timeout and returns
//      false; `expected` arrivals complete a generation, normally the grid)
__device__ __forceinline__ bool grid_barrier(unsigned *count, volatile unsigned *gen, MpDevStatus *st,
                                             bool *abort_s, unsigned long long limit_ns = 1000000000ULL,
                                             unsigned expected = 0) {
    if (expected == 0) expected = gridDim.x;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned g = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(count, 1u);
        if (arrived == expected - 1) {
            *count = 0;
            __threadfence();
            atomicAdd((unsigned *)gen, 1u);
        } else {
            const unsigned long long t0 = global_ns();
            long long polls = 0;
            while (*gen == g) {
                if (++polls > (1LL << 24) || global_ns() - t0 > limit_ns) {
                    mp_flag(st, MP_FLAG_TIMEOUT);
                    atomicExch(&st->timeout_site, 2);
                    *abort_s = true;
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return !*abort_s;
}

// Counts kernel launches (every launch wrapper calls it).
void mp_note_launch(int k = 1);

// Times the launches inside its scope with CUDA events on stream s when
// class cls is enabled in the profiler.
struct MpProfScope {
    int cls;
    double work;
    cudaStream_t s;
    cudaEvent_t e0 = nullptr;
    MpProfScope(int cls_, double work_, cudaStream_t s_);
    ~MpProfScope();
};

// cudaFuncSetAttribute for one kernel on the current device, skipped when
// the same or a larger value was already set there (the host-side cost of the
// call is paid once per kernel, not once per launch).  attr: a
// cudaFuncAttribute; value: its value.
cudaError_t mp_func_attr_once(const void *kern, cudaFuncAttribute attr, int value);
template <typename K>
inline cudaError_t mp_smem_attr(K kern, size_t bytes) {
    return mp_func_attr_once(reinterpret_cast<const void *>(kern), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bytes);
}

static inline int div_up(int a, int b) { return (a + b - 1) / b; }
static inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
