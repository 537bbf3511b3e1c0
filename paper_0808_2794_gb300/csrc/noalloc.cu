// noalloc.cu -- mp_gesv_noalloc: the general solve with its scratch memory in
// a fixed array that lives in this library's device image, for callers that
// are not allowed to allocate device memory.
//
// The array is a file-scope __device__ object, so every GPU that loads this
// library holds its MP_NOALLOC_SCRATCH_BYTES until the process exits.  Host
// code only sees a host-side stand-in under the array's name; the device
// address is looked up once per device with cudaGetSymbolAddress (with that
// device current) and cached here for the life of the process; a device reset
// would reload the module and leave the cached address stale, so the entry
// point is documented as not usable after cudaDeviceReset.
#include <cstdio>
#include <mutex>

#include "common.cuh"
#include "driver.cuh"

static __device__ __align__(256) unsigned char g_noalloc_scratch[MP_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (looked up on first use).
int scratch_address(void **out) {
    int dev = 0;
    MP_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        mp_set_error("mp_gesv_noalloc: device ordinal out of range");
        return -1000 - (int)cudaErrorInvalidDevice;
    }
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        MP_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return 0;
}
}  // namespace

extern "C" size_t mp_noalloc_scratch_bytes(void) { return (size_t)MP_NOALLOC_SCRATCH_BYTES; }

extern "C" int mp_gesv_noalloc(int n, int nrhs, const double *dA, int lda, const double *dB, int ldb,
                               double *dX, int ldx, int32_t *dipiv, const mp_opts *opts, mp_stats *stats,
                               void *stream) {
    if (n >= 0 && nrhs >= 0 && nrhs <= 8) {
        const size_t need = mp_gesv_workspace_bytes(n, nrhs, opts);
        if (need > (size_t)MP_NOALLOC_SCRATCH_BYTES) {
            char msg[200];
            snprintf(msg, sizeof msg,
                     "mp_gesv_noalloc: n=%d nrhs=%d needs %zu bytes of scratch, more than the %zu-byte "
                     "static array; use mp_gesv with a caller workspace",
                     n, nrhs, need, (size_t)MP_NOALLOC_SCRATCH_BYTES);
            return mp_arg_fail(1, msg) ;
        }
    }
    void *scratch = nullptr;
    if (n > 0 && nrhs > 0) {
        int e = scratch_address(&scratch);
        if (e) return e;
    }
    // timing off: the phase timers would create CUDA events
    return mp_gesv_impl(n, nrhs, dA, lda, dB, ldb, dX, ldx, dipiv, scratch, (size_t)MP_NOALLOC_SCRATCH_BYTES,
                        opts, stats, stream, false);
}
