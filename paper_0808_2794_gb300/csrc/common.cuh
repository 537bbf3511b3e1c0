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
