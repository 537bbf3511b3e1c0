// solver.cu -- host driver of the mixed-precision iterative-refinement solver
// and the C ABI declared in include/mpsolve.h.
//
// Algorithm 1 (Section 2.1):
//   1: LU <- PA                 low precision: blocked right-looking LU with a
//                               recursive panel (kernels: panel, row moves,
//                               triangular solve, trailing update)
//   2-3: x_0 from L, U          low precision (blocked triangular solves)
//   do k = 1, 2, ...
//   4:   r_k = b - A x_{k-1}    FP64 with the caller's FP64 A
//        check convergence      normwise backward error per column <= tol
//   5-6: z_k from L, U          low precision, r scaled by a power of two
//   7:   x_k = x_{k-1} + z_k    FP64
// Section 4: when refinement cannot converge (breakdown, stall, iteration
// limit) the solve resorts to a full FP64 LU solve on the GPU.
//
// Every step runs in a CUDA kernel on the caller's stream; the host only
// reads back a small status block once per iteration to decide whether to
// continue.  All scratch memory comes from the caller's workspace.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "common.cuh"
#include "driver.cuh"
#include "kernels.cuh"
#include "tc_gemm.cuh"

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local char g_err[512];

int mp_cuda_fail(cudaError_t e, const char *what, const char *file, int line) {
    snprintf(g_err, sizeof g_err, "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
    return -1000 - (int)e;
}
int mp_arg_fail(int idx, const char *msg) {
    snprintf(g_err, sizeof g_err, "argument %d: %s", idx, msg);
    return -idx;
}
void mp_set_error(const char *msg) { snprintf(g_err, sizeof g_err, "%s", msg); }

extern "C" const char *mp_last_error(void) { return g_err; }

// ---------------------------------------------------------------------------
// instrumentation: launch counter and per-class event timing
// ---------------------------------------------------------------------------
#include <atomic>
#include <mutex>
#include <type_traits>
#include <vector>

static std::atomic<long long> g_launches{0};
void mp_note_launch(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
extern "C" long long mp_launch_count(void) { return g_launches.load(); }

namespace {
struct ProfRec {
    int cls;
    double work;
    cudaEvent_t e0, e1;
};
std::mutex g_prof_mu;
unsigned g_prof_mask = 0;
int g_prof_every = 1;                            // record one scope in every g_prof_every of a class
std::atomic<unsigned> g_prof_seen[MP_KC_COUNT];  // scopes of each class met since the last enable
std::vector<ProfRec> g_prof;
std::vector<cudaEvent_t> g_prof_pool;  // recorded-and-read events, reused (creating one costs host time)

cudaEvent_t prof_event() {
    {
        std::lock_guard<std::mutex> g(g_prof_mu);
        if (!g_prof_pool.empty()) {
            cudaEvent_t e = g_prof_pool.back();
            g_prof_pool.pop_back();
            return e;
        }
    }
    cudaEvent_t e = nullptr;
    return cudaEventCreate(&e) == cudaSuccess ? e : nullptr;
}
// (g_prof_mu held)
void prof_release(const ProfRec &r) {
    g_prof_pool.push_back(r.e0);
    g_prof_pool.push_back(r.e1);
}
}  // namespace

MpProfScope::MpProfScope(int cls_, double work_, cudaStream_t s_) : cls(cls_), work(work_), s(s_) {
    if ((g_prof_mask & (1u << cls)) &&
        (g_prof_every <= 1 || g_prof_seen[cls].fetch_add(1, std::memory_order_relaxed) % g_prof_every == 0)) {
        e0 = prof_event();
        if (e0) cudaEventRecord(e0, s);
    }
}
MpProfScope::~MpProfScope() {
    if (!e0) return;
    cudaEvent_t e1 = prof_event();
    std::lock_guard<std::mutex> g(g_prof_mu);
    if (!e1) {
        g_prof_pool.push_back(e0);
        return;
    }
    cudaEventRecord(e1, s);
    g_prof.push_back({cls, work, e0, e1});
}

cudaError_t mp_func_attr_once(const void *kern, cudaFuncAttribute attr, int value) {
    struct Entry {
        const void *k;
        int attr, dev, value;
    };
    static std::mutex mu;
    static std::vector<Entry> seen;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> g(mu);
    for (auto &x : seen)
        if (x.k == kern && x.attr == (int)attr && x.dev == dev) {
            if (x.value >= value) return cudaSuccess;
            e = cudaFuncSetAttribute(kern, attr, value);
            if (e == cudaSuccess) x.value = value;
            return e;
        }
    e = cudaFuncSetAttribute(kern, attr, value);
    if (e == cudaSuccess) seen.push_back({kern, (int)attr, dev, value});
    return e;
}

extern "C" void mp_profile_enable(unsigned mask) {
    std::lock_guard<std::mutex> g(g_prof_mu);
    for (auto &r : g_prof) {
        cudaEventSynchronize(r.e1);
        prof_release(r);
    }
    g_prof.clear();
    g_prof_mask = mask;
    for (auto &c : g_prof_seen) c.store(0, std::memory_order_relaxed);
}

extern "C" void mp_profile_sample(int every) {
    std::lock_guard<std::mutex> g(g_prof_mu);
    g_prof_every = every < 1 ? 1 : every;
    for (auto &c : g_prof_seen) c.store(0, std::memory_order_relaxed);
}

extern "C" int mp_profile_collect(double *ms, long long *launches, double *work) {
    std::lock_guard<std::mutex> g(g_prof_mu);
    for (int c = 0; c < MP_KC_COUNT; ++c) { ms[c] = 0; launches[c] = 0; work[c] = 0; }
    for (auto &r : g_prof) {
        MP_CUDA_TRY(cudaEventSynchronize(r.e1));
        float t = 0;
        MP_CUDA_TRY(cudaEventElapsedTime(&t, r.e0, r.e1));
        ms[r.cls] += t;
        launches[r.cls] += 1;
        work[r.cls] += r.work;
        prof_release(r);
    }
    g_prof.clear();
    return 0;
}

extern "C" void mp_default_opts(mp_opts *o) {
    o->prec = MP_PREC_FP32;
    o->refine = MP_REFINE_CLASSICAL;
    o->itermax = 30;
    o->tol = 1e-14;
    o->gmres_restart = 30;
    o->gmres_tol = 1e-6;
    o->stall_ratio = 0.5;
    o->allow_fallback = 1;
    o->nb_outer = 0;
    o->nb_inner = 0;
}

extern "C" int mp_factor_ld(int n) { return std::max(32, (n + 31) / 32 * 32); }

namespace {

constexpr int kMaxRhs = 8;

// Status block in device memory, read back by the host once per iteration.
struct StatusBlock {
    MpDevStatus st;
    double pad0;
    double bnorm[kMaxRhs];
    double rnorm[kMaxRhs];
    double xnorm[kMaxRhs];
    double znorm[kMaxRhs];
    double rr[kMaxRhs];  // ||r_c||_2^2 for the GMRES cycles
    MpDevStatus gst;     // status sink for the GMRES basis scans (not the input's)
    int factor_kind;     // factors left in the workspace by the last solve (FactorKind)
    int pad1;
};

// What a finished mp_gesv / mp_posv leaves in its workspace, for the adjoint.
enum FactorKind { kNoFactors = 0, kLuF32 = 1, kLuF64 = 2, kCholF32 = 3, kCholF64 = 4 };

int outer_nb(int n, const mp_opts &o) {
    if (o.nb_outer > 0) return std::min(1024, std::max(32, o.nb_outer / 32 * 32));
    // wider panels make the tensor-core trailing update more efficient, but
    // the leaf pipeline's bulk launches (which also form U12 left-looking,
    // K up to the panel width) then outgrow the panel kernels they overlap
    if (o.prec == MP_PREC_FP32 || o.prec == MP_PREC_FP64) return n >= 4096 ? 256 : 128;
    return n >= 8192 ? 384 : 256;
}

// ---------------------------------------------------------------------------
// workspace layout
// ---------------------------------------------------------------------------
struct Layout {
    size_t status, rowsum, W, perm, ipiv, pairs, npairs, map, Linv, Uinv, invtmp, acc, bar, R, Y, Z,
        part, tc, linv, gV, gZ, gsm, total;
    size_t W_bytes;
    int ldw, nblk, ksplit, nb;
};

size_t carve(size_t &off, size_t bytes) {
    off = align_up(off, 256);
    const size_t at = off;
    off += bytes;
    return at;
}

// Room for FP64 factors is needed by the fallback and by the plain FP64 solve.
bool fp64_space_of(const mp_opts &o) { return o.allow_fallback != 0 || o.prec == MP_PREC_FP64; }

// fp64_space: room for the FP64 fallback (W, inverses, vectors sized for double)
Layout make_layout(int n, int nrhs, const mp_opts &o, bool fp64_space, bool sym = false) {
    Layout L{};
    L.ldw = mp_factor_ld(n);
    L.nblk = (n + 63) / 64;  // blocks of the FP64 solve (the FP32 solve uses half as many)
    L.ksplit = residual_ksplit(n, nrhs);
    L.nb = outer_nb(n, o);
    const size_t el = fp64_space ? sizeof(double) : sizeof(float);
    const int rhs = std::max(nrhs, 1);
    size_t off = 0;
    L.status = carve(off, sizeof(StatusBlock));
    L.rowsum = carve(off, sizeof(double) * (size_t)n);
    L.W_bytes = (size_t)n * (size_t)L.ldw * el;
    L.W = carve(off, L.W_bytes);
    L.perm = carve(off, sizeof(int) * (size_t)n);
    L.ipiv = carve(off, sizeof(int) * (size_t)n);
    L.pairs = carve(off, sizeof(int2) * ((size_t)2 * (size_t)std::max(n, L.nb) + 128));  // + two leaves' moves
    L.npairs = carve(off, sizeof(int) * 32);  // [0], [1]: two leaves' move counts, [2]: max |U12|, [4..20): tickets
    L.map = carve(off, sizeof(int) * (size_t)n);
    const size_t inv_bytes = std::max(trsv_inverse_bytes<float>(n), fp64_space ? trsv_inverse_bytes<double>(n) : 0);
    L.Linv = carve(off, inv_bytes);
    L.Uinv = carve(off, inv_bytes);
    L.invtmp = carve(off, std::max(trsv_tmp_bytes<float>(n), fp64_space ? trsv_tmp_bytes<double>(n) : 0));
    L.acc = carve(off, el * (size_t)n * rhs);
    L.bar = carve(off, std::max(trsv_sync_bytes<float>(n), fp64_space ? trsv_sync_bytes<double>(n) : 0));
    L.R = carve(off, sizeof(double) * (size_t)n * rhs);
    L.Y = carve(off, el * (size_t)n * rhs);
    L.Z = carve(off, el * (size_t)n * rhs);
    if (sym) L.ksplit = residual_sym_blocks(n);  // the symmetric residual's partial sums
    L.part = carve(off, sizeof(double) * (size_t)L.ksplit * n * rhs);
    L.tc = carve(off, o.prec == MP_PREC_FP32 || o.prec == MP_PREC_FP64
                          ? 0
                          : std::max(tc_workspace_bytes(n, L.nb, o.prec),
                                                        tc_workspace_bytes(n, L.nb, MP_PREC_FP16X3)));
    L.linv = carve(off, 3 * 1024 * sizeof(double));  // three leaves' L11^{-1}
    // GMRES: Krylov basis V (m+1 columns), preconditioned vectors Z (m), small vectors
    const size_t m = o.refine == MP_REFINE_CLASSICAL ? 0 : (size_t)std::max(o.gmres_restart, 1);
    L.gV = carve(off, m ? sizeof(double) * (size_t)n * (m + 1) : 0);
    L.gZ = carve(off, sizeof(double) * (size_t)n * m);
    L.gsm = carve(off, m ? sizeof(double) * (3 * m + 8) : 0);
    L.total = align_up(off, 256);
    return L;
}

template <typename P>
P *at(void *work, size_t off) {
    return reinterpret_cast<P *>(static_cast<char *>(work) + off);
}

__global__ void iota_kernel(int *v, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) v[i] = i;
}
cudaError_t launch_iota(int *v, int n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    mp_note_launch();
    iota_kernel<<<std::min(1024, (n + 255) / 256), 256, 0, s>>>(v, n);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// factorization
// ---------------------------------------------------------------------------
template <typename T>
struct FactorCtx {
    T *W;
    long ld;
    int n;
    int32_t *ipiv;
    int *perm;
    int2 *pairs;
    int *npairs;
    int *map;
    MpDevStatus *st;
    cudaStream_t s;
    int prec;
    void *tc;
    T *linv;  // inverse of the last leaf's L11 (panel_base_width^2 elements)
};

#define CU(expr)                                      \
    do {                                              \
        cudaError_t _e = (expr);                      \
        if (_e != cudaSuccess) return _e;             \
    } while (0)

// C -= A B for the FP32-accurate updates inside the panel and the triangular
// solve: plain FP32 FMA for the FP32 rung (and in FP64 for the fallback),
// the split-fp16 tensor-core product (about FP32 accuracy) for the tensor-core
// rungs, once the product is large enough to fill the machine.
template <typename T>
cudaError_t gemm_fp32_accurate(FactorCtx<T> &c, int M, int N, int K, const T *A, long lda, const T *B, long ldb,
                               T *C, long ldc) {
    if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
    if (sizeof(T) == 4 && c.prec != MP_PREC_FP32 && (double)M * N * K >= 1.0e8 && lda % 4 == 0 && ldb % 4 == 0)
        return tc_trailing_update(MP_PREC_FP16X3, M, N, K, reinterpret_cast<const float *>(A), lda,
                                  reinterpret_cast<const float *>(B), ldb, reinterpret_cast<float *>(C), ldc, c.tc,
                                  c.st, c.s);
    return launch_gemm_sub<T>(M, N, K, A, lda, B, ldb, C, ldc, c.s);
}

// B <- L^{-1} B, L unit lower m x m (recursive: small base solve + GEMM update).
template <typename T>
cudaError_t trsm_rec(FactorCtx<T> &c, int m, int N, const T *L, long ldl, T *B, long ldb) {
    if (m <= 0 || N <= 0) return cudaSuccess;
    if (m <= 64) return launch_trsm_llnu_small<T>(m, N, L, ldl, B, ldb, c.s);
    const int m1 = (m / 2 + 31) / 32 * 32;
    CU(trsm_rec<T>(c, m1, N, L, ldl, B, ldb));
    CU(gemm_fp32_accurate<T>(c, m - m1, N, m1, L + (long)m1 * ldl, ldl, B, ldb, B + (long)m1 * ldb, ldb));
    return trsm_rec<T>(c, m - m1, N, L + (long)m1 * ldl + m1, ldl, B + (long)m1 * ldb, ldb);
}

// Per-device pair of internal streams for the panel: a high-priority one for
// the chain of leaves and a low-priority one for the bulk of each leaf's
// update (created once).
struct PanelStreams {
    cudaStream_t hi = nullptr, lo = nullptr;
};
PanelStreams panel_streams() {
    static std::mutex mu;
    static PanelStreams per_dev[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return PanelStreams{};
    std::lock_guard<std::mutex> g(mu);
    PanelStreams &p = per_dev[dev];
    if (!p.hi) {
        int lo_pri = 0, hi_pri = 0;
        if (cudaDeviceGetStreamPriorityRange(&lo_pri, &hi_pri) != cudaSuccess ||
            cudaStreamCreateWithPriority(&p.hi, cudaStreamNonBlocking, hi_pri) != cudaSuccess ||
            cudaStreamCreateWithPriority(&p.lo, cudaStreamNonBlocking, lo_pri) != cudaSuccess)
            p = PanelStreams{};
    }
    return p;
}

// LU of the outer panel, columns [k0, k0+ncols) of rows [k0, n), leaf by
// leaf (right-looking inside the panel).  A leaf of at most the base width is
// one cluster panel kernel (which also leaves L11^{-1} and its row moves);
// the leaf's row exchange and the fused U-block + update of the panel's
// columns right of it follow (FP32 FMA; FP64 in the fallback).
// Leaf-level look-ahead, on two internal streams: the chain (high priority)
// is the sequence of panel kernels, each of which first applies the previous
// leaf's row moves and update to its own columns as it loads them.  The rest
// of each leaf's work -- the update of the columns after the next leaf's, the
// exchange of the columns outside the outer panel and of the row permutation
// -- is one persistent launch on a low-priority stream, shaped in clusters so
// that the next panel kernel always finds a free cluster slot beside it.  A
// panel kernel waits for the bulk launch of two leaves before.  L11^{-1} and
// the moves of two consecutive leaves live in alternating buffers.
template <typename T>
cudaError_t getrf_panel(FactorCtx<T> &c, int k0, int ncols, bool *u12_done, unsigned **u12_max) {
    T *W = c.W;
    const long ld = c.ld;
    unsigned *ticket = reinterpret_cast<unsigned *>(c.npairs + 4);  // one per 128-column chunk
    *u12_done = false;
    if (u12_max) *u12_max = nullptr;
    PanelStreams ps_ = panel_streams();
    cudaEvent_t ev_in = nullptr, ev_chain = nullptr, ev_rest[2] = {nullptr, nullptr};
    bool two = ps_.hi && ps_.lo && ncols > 2 * panel_base_width<T>(c.n - k0) &&
               leaf_update_rest_clusters<T>(panel_cluster_size<T>(c.n - k0)) > 0;
    if (two && (cudaEventCreateWithFlags(&ev_in, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&ev_chain, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&ev_rest[0], cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&ev_rest[1], cudaEventDisableTiming) != cudaSuccess)) {
        two = false;
    }
    cudaStream_t user = c.s, hi = two ? ps_.hi : c.s, lo = two ? ps_.lo : c.s;
    cudaError_t err = cudaSuccess;
    auto chk = [&](cudaError_t e) { if (err == cudaSuccess && e != cudaSuccess) err = e; return err == cudaSuccess; };
    if (two) {
        chk(cudaEventRecord(ev_in, user));
        chk(cudaStreamWaitEvent(hi, ev_in, 0));
        chk(cudaStreamWaitEvent(lo, ev_in, 0));
    }
    const int tc0 = k0 + ncols, tc1 = c.n;  // the trailing columns
    // max |U12| for the scaled tensor-core rungs, raised as U12 is formed
    unsigned *umax = (two && sizeof(T) == 4 && c.prec != MP_PREC_FP32 && tc1 > tc0)
                         ? reinterpret_cast<unsigned *>(c.npairs + 2)
                         : nullptr;
    // zeroed on the bulk stream, ahead of every launch that raises it
    if (umax && err == cudaSuccess) chk(cudaMemsetAsync(umax, 0, sizeof(unsigned), lo));
    c.s = hi;
    int leaf = 0, kb_prev = 0, xs_prev = 0, k_prev = 0;
    for (int k = k0; k < k0 + ncols && err == cudaSuccess; ++leaf) {
        const int m = c.n - k;
        const int kb = std::min(panel_base_width<T>(m), k0 + ncols - k);
        const int xs = panel_base_width<T>(m);
        const int N = k0 + ncols - k - kb;
        // this leaf's L11^{-1} (three buffers: the bulk launch of the next
        // leaf still reads it while the leaf after that is factored) and row
        // moves (two buffers)
        T *X = c.linv + (leaf % 3) * 1024;
        T *Xprev = c.linv + ((leaf + 2) % 3) * 1024;
        int2 *pairs = c.pairs + (leaf & 1) * 64;
        int *npairs = c.npairs + (leaf & 1);
        if (!two) {
            {
                MpProfScope ps(MP_KC_PANEL, (double)m * kb * kb - (double)kb * kb * kb / 3.0, hi);
                if (!chk(launch_panel<T>(W + (long)k * ld + k, ld, m, kb, k, c.ipiv + k, pairs, npairs, c.st, X,
                                         PanelPrev<T>{}, hi)))
                    break;
            }
            {
                MpProfScope ps(MP_KC_ROWMOVES, 4.0 * kb * (double)(c.n - kb) * sizeof(T), hi);
                if (!chk(launch_apply_moves<T>(W, ld, pairs, npairs, 2 * kb, 0, k, k + kb, c.n, c.perm, hi))) break;
            }
            if (N > 0) {
                MpProfScope ps(MP_KC_PANELGEMM, (double)kb * kb * N + 2.0 * (m - kb) * N * kb, hi);
                chk(launch_leaf_update<T>(W, ld, k, kb, 0, N, m - kb, X, xs, ticket, hi));
            }
        } else {
            // the bulk launch of leaf - 2 has brought these columns up to date
            // (and released this parity's buffers); the previous leaf's moves
            // and update are applied by the panel kernel as it loads them
            if (leaf >= 2 && !chk(cudaStreamWaitEvent(hi, ev_rest[leaf & 1], 0))) break;
            PanelPrev<T> pv;
            if (leaf >= 1) {
                pv.X = Xprev;
                pv.pairs = c.pairs + ((leaf - 1) & 1) * 64;
                pv.npairs = c.npairs + ((leaf - 1) & 1);
                pv.xs = xs_prev;
                pv.kb = kb_prev;
            }
            {
                MpProfScope ps(MP_KC_PANEL, (double)m * kb * kb - (double)kb * kb * kb / 3.0, hi);
                if (!chk(launch_panel<T>(W + (long)k * ld + k, ld, m, kb, k, c.ipiv + k, pairs, npairs, c.st, X, pv,
                                         hi)))
                    break;
            }
            if (!chk(cudaEventRecord(ev_chain, hi))) break;
            if (!chk(cudaStreamWaitEvent(lo, ev_chain, 0))) break;
            // the bulk: the columns after the next leaf's, the exchange of the
            // columns outside the outer panel and of the row permutation, and
            // the previous leaf's U rows over the trailing columns; in
            // clusters of the next panel's size, leaving one such cluster free
            const int kb_next = N > 0 ? std::min(panel_base_width<T>(m - kb), N) : 0;
            const int cl = panel_cluster_size<T>(std::max(1, m - kb));
            const int G = leaf_update_rest_clusters<T>(cl);
            LeafRestArgs<T> ra;
            ra.W = W;
            ra.ld = ld;
            ra.k = k;
            ra.kb = kb;
            ra.coff = kb_next;
            ra.N = N - kb_next;
            ra.M = m - kb;
            ra.X = X;
            ra.xs = xs;
            ra.tickets = ticket + 8;
            ra.pairs = pairs;
            ra.npairs = npairs;
            ra.mc1 = k;
            ra.mc2 = tc0;
            ra.mc3 = tc1;
            ra.perm = c.perm;
            if (leaf >= 1 && tc1 > tc0) {
                ra.Xp = Xprev;
                ra.xps = xs_prev;
                ra.kp = k_prev;
                ra.kbp = kb_prev;
                ra.k0 = k0;
                ra.tc0 = tc0;
                ra.tc1 = tc1;
                ra.umax = umax;
            }
            MpProfScope ps(MP_KC_PANELGEMM,
                           (double)kb * kb * (N - kb_next) + 2.0 * (m - kb) * (N - kb_next) * kb +
                               2.0 * (double)ra.kbp * (tc1 - tc0) * (k_prev - k0 + ra.kbp),
                           lo);
            if (!chk(launch_leaf_rest<T>(ra, std::max(1, G), cl, lo))) break;
            if (!chk(cudaEventRecord(ev_rest[leaf & 1], lo))) break;
        }
        kb_prev = kb;
        xs_prev = xs;
        k_prev = k;
        k += kb;
    }
    if (two && err == cudaSuccess && tc1 > tc0) {
        // the last leaf's U rows over the trailing columns
        LeafRestArgs<T> ra;
        ra.W = W;
        ra.ld = ld;
        ra.Xp = c.linv + ((leaf + 2) % 3) * 1024;
        ra.xps = xs_prev;
        ra.kp = k_prev;
        ra.kbp = kb_prev;
        ra.k0 = k0;
        ra.tc0 = tc0;
        ra.tc1 = tc1;
        ra.umax = umax;
        const int G = leaf_update_rest_clusters<T>(1);
        MpProfScope ps(MP_KC_PANELGEMM, 2.0 * (double)kb_prev * (tc1 - tc0) * (k_prev - k0 + kb_prev), lo);
        chk(launch_leaf_rest<T>(ra, std::max(1, G), 1, lo));
    }
    c.s = user;
    if (two) {
        chk(cudaEventRecord(ev_chain, hi));
        chk(cudaStreamWaitEvent(user, ev_chain, 0));
        chk(cudaEventRecord(ev_rest[0], lo));
        chk(cudaStreamWaitEvent(user, ev_rest[0], 0));
        cudaEventDestroy(ev_in);
        cudaEventDestroy(ev_chain);
        cudaEventDestroy(ev_rest[0]);
        cudaEventDestroy(ev_rest[1]);
        *u12_done = err == cudaSuccess && tc1 > tc0;
        if (u12_max) *u12_max = *u12_done ? umax : nullptr;
    }
    return err;
}

// Blocked right-looking LU: panel of width nb (recursive, rows exchanged over
// the whole matrix as each leaf finishes), U12 = L11^{-1} A12, A22 -= L21 U12
// at precision prec.
template <typename T>
cudaError_t getrf_blocked(FactorCtx<T> &c, int nb) {
    const int n = c.n;
    T *W = c.W;
    const long ld = c.ld;
    CU(cudaMemsetAsync(c.npairs + 4, 0, 16 * sizeof(int), c.s));  // the leaf-update tickets (two sets)
    for (int k = 0; k < n; k += nb) {
        const int nbk = std::min(nb, n - k);
        bool u12_done = false;  // U12 formed leaf by leaf during the panel
        unsigned *u12_max = nullptr;  // and its max |.|, when taken on the way
        CU(getrf_panel<T>(c, k, nbk, &u12_done, &u12_max));
        const int rest = n - k - nbk;
        if (rest > 0) {
            if (!u12_done) {
                MpProfScope ps(MP_KC_TRSM, (double)nbk * nbk * rest, c.s);
                CU(trsm_rec<T>(c, nbk, rest, W + (long)k * ld + k, ld, W + (long)k * ld + k + nbk, ld));
            }
            MpProfScope ps(MP_KC_UPDATE, 2.0 * rest * rest * nbk, c.s);
            const T *L21 = W + (long)(k + nbk) * ld + k;
            const T *U12 = W + (long)k * ld + k + nbk;
            T *A22 = W + (long)(k + nbk) * ld + k + nbk;
            if (sizeof(T) == 4 && c.prec != MP_PREC_FP32) {
                CU(tc_trailing_update(c.prec, rest, rest, nbk, reinterpret_cast<const float *>(L21), ld,
                                      reinterpret_cast<const float *>(U12), ld,
                                      reinterpret_cast<float *>(A22), ld, c.tc, c.st, c.s, u12_max));
            } else {
                CU(launch_gemm_sub<T>(rest, rest, nbk, L21, ld, U12, ld, A22, ld, c.s));
            }
        }
    }
    return cudaSuccess;
}

// C -= A B^T for the Cholesky updates inside the recursive panel, with the
// same choice of arithmetic as gemm_fp32_accurate.  lower: only the tiles on
// or below the diagonal of C (its top square is a diagonal block).
template <typename T>
cudaError_t gemm_nt_fp32_accurate(FactorCtx<T> &c, int M, int N, int K, const T *A, long lda, const T *B,
                                  long ldb, T *C, long ldc, int lower) {
    if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
    if (sizeof(T) == 4 && c.prec != MP_PREC_FP32 && (double)M * N * K >= 1.0e8 && lda % 4 == 0 && ldb % 4 == 0)
        return tc_update_nt(MP_PREC_FP16X3, M, N, K, reinterpret_cast<const float *>(A), lda,
                            reinterpret_cast<const float *>(B), ldb, reinterpret_cast<float *>(C), ldc, lower, c.tc,
                            c.st, c.s);
    return launch_gemm_nt_sub<T>(M, N, K, A, lda, B, ldb, C, ldc, lower, c.s);
}

// Recursive Cholesky of columns [k0, k0+ncols) of rows [k0, n) (Section
// 3.1.1, SPOTRF; lower, A = L L^T): left half, then the right half's columns
// are updated with the left half's L (A -= L_left L_top^T), right half.  A
// leaf (ncols <= leaf width) factors its diagonal block and solves the rows
// below it in one launch.
template <typename T>
cudaError_t potrf_rec(FactorCtx<T> &c, int k0, int ncols) {
    const int m = c.n - k0;
    const int leaf = potrf_leaf_width();
    T *W = c.W;
    const long ld = c.ld;
    if (ncols <= leaf) {
        MpProfScope ps(MP_KC_PANEL, (double)m * ncols * ncols - 2.0 * ncols * ncols * ncols / 3.0, c.s);
        return launch_potrf_leaf<T>(c.n, k0, ncols, W, ld, c.st, c.s);
    }
    int n1 = (ncols / 2) / leaf * leaf;
    if (n1 < leaf) n1 = leaf;
    CU(potrf_rec<T>(c, k0, n1));
    {
        MpProfScope ps(MP_KC_PANELGEMM, 2.0 * (m - n1) * (ncols - n1) * n1, c.s);
        CU(gemm_nt_fp32_accurate<T>(c, m - n1, ncols - n1, n1, W + (long)(k0 + n1) * ld + k0, ld,
                                    W + (long)(k0 + n1) * ld + k0, ld, W + (long)(k0 + n1) * ld + k0 + n1, ld, 1));
    }
    return potrf_rec<T>(c, k0 + n1, ncols - n1);
}

// Blocked right-looking Cholesky: panel of width nb (recursive), then the
// trailing update A22 -= fl_p(L21) fl_p(L21)^T on the lower tiles, at
// precision prec (the symmetric rank-nb update, SSYRK's place in SPOTRF).
template <typename T>
cudaError_t potrf_blocked(FactorCtx<T> &c, int nb) {
    const int n = c.n;
    T *W = c.W;
    const long ld = c.ld;
    for (int k = 0; k < n; k += nb) {
        const int nbk = std::min(nb, n - k);
        CU(potrf_rec<T>(c, k, nbk));
        const int rest = n - k - nbk;
        if (rest > 0) {
            MpProfScope ps(MP_KC_UPDATE, (double)rest * rest * nbk, c.s);
            const T *L21 = W + (long)(k + nbk) * ld + k;
            T *A22 = W + (long)(k + nbk) * ld + k + nbk;
            if (sizeof(T) == 4 && c.prec != MP_PREC_FP32) {
                CU(tc_update_nt(c.prec, rest, rest, nbk, reinterpret_cast<const float *>(L21), ld,
                                reinterpret_cast<const float *>(L21), ld, reinterpret_cast<float *>(A22), ld, 1,
                                c.tc, c.st, c.s));
            } else {
                CU(launch_gemm_nt_sub<T>(rest, rest, nbk, L21, ld, L21, ld, A22, ld, 1, c.s));
            }
        }
    }
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// the solve
// ---------------------------------------------------------------------------
struct Solve {
    int n, nrhs;
    const double *A;
    int lda;
    const double *B;
    int ldb;
    double *X;
    int ldx;
    void *work;
    Layout L;
    cudaStream_t s;
    StatusBlock *sb;
    int epoch;
    bool sym;    // symmetric positive definite A, lower triangle (Cholesky)
    bool trans;  // adjoint solve A^T x = b with the transposed LU factors below
    void *tW, *tLinv, *tUinv;  // W^T (row-major, ld S.L.ldw) and its diagonal-block inverses
};

int read_status(Solve &S, StatusBlock &h) {
    MP_CUDA_TRY(cudaMemcpyAsync(&h, S.sb, sizeof(StatusBlock), cudaMemcpyDeviceToHost, S.s));
    MP_CUDA_TRY(cudaStreamSynchronize(S.s));
    return 0;
}

// z = U^{-1} L^{-1} P (r / s) in T for nrhs columns of the FP64 R (rnorm
// gives s); result in S.Z.
// With S.trans the factors are those of A^T = U^T L^T P: W^T holds U^T
// (lower, non-unit) and L^T (upper, unit), the row permutation is applied
// after the solve (by the update's scatter) instead of before it.
template <typename T>
int lowp_solve(Solve &S, const double *R, long ldr, const double *rnorm, int nrhs) {
    const Layout &L = S.L;
    T *W = S.trans ? static_cast<T *>(S.tW) : at<T>(S.work, L.W);
    const T *Linv = S.trans ? static_cast<const T *>(S.tLinv) : at<T>(S.work, L.Linv);
    const T *Uinv = S.trans ? static_cast<const T *>(S.tUinv) : at<T>(S.work, L.Uinv);
    const int *perm = S.trans ? nullptr : at<int>(S.work, L.perm);
    ++S.epoch;
    MpProfScope ps(MP_KC_TRSV, (double)S.n * S.n * sizeof(T) + 4.0 * S.n * nrhs * sizeof(T), S.s);
    MP_CUDA_TRY(launch_trsv_lower<T>(S.n, nrhs, W, L.ldw, Linv, R, ldr, perm, rnorm, at<T>(S.work, L.Y), S.n,
                                     at<T>(S.work, L.acc), at<unsigned>(S.work, L.bar), &S.sb->st, S.s));
    MP_CUDA_TRY(launch_trsv_upper<T>(S.n, nrhs, W, L.ldw, Uinv, at<T>(S.work, L.Y), S.n, at<T>(S.work, L.Z), S.n,
                                     at<T>(S.work, L.acc), at<unsigned>(S.work, L.bar), &S.sb->st, S.s));
    return 0;
}

// Row permutation applied to a correction before it is added (adjoint only).
const int *update_scatter(Solve &S) { return S.trans ? at<int>(S.work, S.L.perm) : nullptr; }

// R = B - A X (R = A X when B is null) for nrhs columns in FP64, with
// rnorm/xnorm (zeroed by the caller): the general product, or the
// symmetric one reading the lower triangle of A only.
int apply_A(Solve &S, int nrhs, const double *X, long ldx, const double *B, long ldb, double *R, long ldr,
            double *rnorm, double *xnorm, MpDevStatus *st) {
    const Layout &L = S.L;
    const double bytes = (S.sym ? 4.0 : 8.0) * S.n * S.n + 32.0 * S.n * nrhs;
    MpProfScope ps(MP_KC_RESIDUAL, bytes, S.s);
    int ks;
    if (S.trans) {  // adjoint: R = B - A^T X, column dots of A (B is never null here)
        MP_CUDA_TRY(launch_residual_trans(S.n, nrhs, S.A, S.lda, X, ldx, B, ldb, R, ldr, rnorm, xnorm, st, S.s));
        return 0;
    }
    if (S.sym) {
        ks = residual_sym_blocks(S.n);
        MP_CUDA_TRY(launch_residual_sym_partial(S.n, nrhs, S.A, S.lda, X, ldx, at<double>(S.work, L.part), S.s));
    } else {
        ks = nrhs == S.nrhs ? L.ksplit : residual_ksplit(S.n, nrhs);
        MP_CUDA_TRY(launch_residual_partial(S.n, nrhs, S.A, S.lda, X, ldx, at<double>(S.work, L.part), ks, S.s));
    }
    MP_CUDA_TRY(launch_residual_finalize(S.n, nrhs, at<double>(S.work, L.part), ks, B, ldb, X, ldx, R, ldr, rnorm,
                                         xnorm, st, S.s));
    return 0;
}

int residual(Solve &S) {
    MP_CUDA_TRY(cudaMemsetAsync(S.sb->rnorm, 0, sizeof(double) * 2 * kMaxRhs, S.s));  // rnorm, xnorm
    return apply_A(S, S.nrhs, S.X, S.ldx, S.B, S.ldb, at<double>(S.work, S.L.R), S.n, S.sb->rnorm, S.sb->xnorm,
                   &S.sb->st);
}

// Resets the grid-barrier words of the triangular solves.
int reset_sync(Solve &S) {
    MP_CUDA_TRY(cudaMemsetAsync(at<unsigned>(S.work, S.L.bar), 0, sizeof(unsigned) * 4, S.s));
    S.epoch = 0;
    return 0;
}

// Factor (T = float: low precision; T = double: fallback) and leave factors,
// perm and diagonal inverses in the workspace.  Returns the zero-pivot info.
template <typename T>
int factor(Solve &S, int prec, int nb, int *info_out, uint32_t *flags_out) {
    const Layout &L = S.L;
    T *W = at<T>(S.work, L.W);
    MP_CUDA_TRY(launch_iota(at<int>(S.work, L.perm), S.n, S.s));
    MP_CUDA_TRY(launch_iota(at<int>(S.work, L.map), S.n, S.s));
    FactorCtx<T> c{W, (long)L.ldw, S.n, at<int32_t>(S.work, L.ipiv), at<int>(S.work, L.perm),
                   at<int2>(S.work, L.pairs), at<int>(S.work, L.npairs), at<int>(S.work, L.map),
                   &S.sb->st, S.s, prec, at<void>(S.work, L.tc), at<T>(S.work, L.linv)};
    if (S.sym) {
        // A = L L^T; L^T mirrored into the upper triangle; the lower solve
        // uses L's own (non-unit) diagonal
        MP_CUDA_TRY(potrf_blocked<T>(c, nb));
        MP_CUDA_TRY(launch_mirror_lower<T>(S.n, W, L.ldw, S.s));
        MP_CUDA_TRY(launch_build_inverses<T>(S.n, W, L.ldw, at<T>(S.work, L.Linv), at<T>(S.work, L.Uinv),
                                             at<T>(S.work, L.invtmp), S.s, false));
    } else {
        MP_CUDA_TRY(getrf_blocked<T>(c, nb));
        MP_CUDA_TRY(launch_build_inverses<T>(S.n, W, L.ldw, at<T>(S.work, L.Linv), at<T>(S.work, L.Uinv),
                                             at<T>(S.work, L.invtmp), S.s));
    }
    StatusBlock h;
    int e = read_status(S, h);
    if (e) return e;
    *info_out = h.st.zero_pivot;
    *flags_out = h.st.flags;
    return 0;
}

double bwd_of(const StatusBlock &h, int c) {
    const double den = h.st.anorm * h.xnorm[c] + h.bnorm[c];
    if (!(h.rnorm[c] == h.rnorm[c])) return INFINITY;
    return den > 0.0 ? h.rnorm[c] / den : (h.rnorm[c] > 0.0 ? INFINITY : 0.0);
}

// Refinement loop with the factors of precision T (Algorithm 1 steps 2-7).
// x_k is accepted when every column has bwd <= tol AND has reached the FP64
// floor (bwd == 0; bwd <= 2 u64, which bounds the forward error by
// 2 kappa bwd <= 4 kappa u64; last correction <= 4 u64 ||x_k||; or the
// corrections stopped shrinking); the shrink test with bwd > tol is a stall.
// Returns 0, or a CUDA error code; *conv tells whether all columns converged.
template <typename T>
int refine(Solve &S, const mp_opts &o, int itermax, bool stall_test, mp_stats *st, bool *conv,
           int *iters, uint32_t *flags) {
    StatusBlock h;
    // steps 2-3: x_0 from b (scaled by 2^ceil(log2 ||b||)); znorm = ||x_0||
    MP_CUDA_TRY(cudaMemsetAsync(S.sb->znorm, 0, sizeof(double) * kMaxRhs, S.s));
    int e = lowp_solve<T>(S, S.B, S.ldb, S.sb->bnorm, S.nrhs);
    if (e) return e;
    MP_CUDA_TRY(launch_update<T>(S.n, S.nrhs, at<T>(S.work, S.L.Z), S.n, S.sb->bnorm, S.X, S.ldx,
                                 S.sb->znorm, 1, S.s, update_scatter(S)));
    double zprev[kMaxRhs] = {0};
    int it = 0;
    *conv = false;
    const double u64 = 1.1102230246251565e-16;
    for (;;) {
        if ((e = residual(S))) return e;
        if ((e = read_status(S, h))) return e;
        double worst = 0.0;
        bool done = true, nonfinite = false, stalled = false, all_tol = true;
        for (int c = 0; c < S.nrhs; ++c) {
            const double b = bwd_of(h, c);
            const bool stagnant = it >= 2 && h.znorm[c] > o.stall_ratio * zprev[c];
            const bool at_floor = b == 0.0 || b <= 2.0 * u64 || h.znorm[c] <= 4.0 * u64 * h.xnorm[c] || stagnant;
            if (!(b <= o.tol)) all_tol = false;
            if (!(b <= o.tol && at_floor)) done = false;
            if (!(b <= o.tol) && stagnant) stalled = true;
            if (!(b == b) || std::isinf(b)) nonfinite = true;
            worst = std::max(worst, std::isnan(b) ? INFINITY : b);
        }
        if (st) {
            if (st->nhist < 32) st->hist[st->nhist++] = worst;
            st->bwd_err = worst;
        }
        *flags |= h.st.flags & (MP_FLAG_TIMEOUT | MP_FLAG_NONFINITE_INPUT);
        if (h.st.flags & MP_FLAG_TIMEOUT) break;
        if (nonfinite) { *flags |= MP_FLAG_LOWP_BREAKDOWN; break; }
        if (done) { *conv = true; break; }
        if (stalled && stall_test) { *flags |= MP_FLAG_STALLED; break; }
        if (it >= itermax) { *conv = all_tol; break; }
        std::memcpy(zprev, h.znorm, sizeof zprev);
        // steps 5-7
        if ((e = lowp_solve<T>(S, at<double>(S.work, S.L.R), S.n, S.sb->rnorm, S.nrhs))) return e;
        MP_CUDA_TRY(cudaMemsetAsync(S.sb->znorm, 0, sizeof(double) * kMaxRhs, S.s));
        MP_CUDA_TRY(launch_update<T>(S.n, S.nrhs, at<T>(S.work, S.L.Z), S.n, S.sb->rnorm, S.X, S.ldx,
                                     S.sb->znorm, 0, S.s, update_scatter(S)));
        if (st) st->n_precond += 1;
        ++it;
    }
    *iters = it;
    return 0;
}

// ---------------------------------------------------------------------------
// GMRES-based refinement (Section 2.2, Eq. 2; Section 4): the correction
// equation A d = r is solved by one cycle of right-preconditioned GMRES with
// M = (LU)^{-1} P from the low-precision factors, in the flexible form that
// keeps the preconditioned vectors z_k = M v_k (so x += Z y needs no further
// application of M).  The Arnoldi process runs in FP64 on the device; the
// (m+1) x m Hessenberg matrix, its Givens rotations and the small triangular
// solve stay on the host (m <= a few dozen).  Orthogonalisation is classical
// Gram-Schmidt applied twice (one reduction and one update per pass instead of
// k dependent ones), which matches modified Gram-Schmidt's loss of
// orthogonality at O(u) for the basis sizes used here.
// ---------------------------------------------------------------------------
struct GmresScratch {
    double *V, *Z, *h1, *h2, *hh, *vnorm, *tn, *y;
};

GmresScratch gmres_scratch(Solve &S, int m) {
    double *g = at<double>(S.work, S.L.gsm);
    GmresScratch G;
    G.V = at<double>(S.work, S.L.gV);
    G.Z = at<double>(S.work, S.L.gZ);
    G.h1 = g;
    G.h2 = g + (m + 1);
    G.hh = g + 2 * (m + 1);
    G.vnorm = G.hh + 1;
    G.tn = G.vnorm + 1;  // two scratch norms of A z
    G.y = G.tn + 2;      // m entries
    return G;
}

// One GMRES cycle on A d = r_c (r_c = column c of the FP64 residual in
// S.L.R, beta = ||r_c||_2 > 0); applies x_c += Z y and leaves ||Z y||inf in
// sb->znorm[c] (zeroed by the caller).  *steps = inner steps taken; *bad is
// set when the Arnoldi process produced a non-finite value.
// The inner loop stops once the least-squares residual |g_k| is below
// gmres_tol * beta or below sqrt(n) u64 ||A||inf ||x_c||inf (floor), the
// level at which r itself is known.
template <typename T>
int gmres_cycle(Solve &S, const mp_opts &o, int c, double beta, double floor, int *steps, bool *bad) {
    const int n = S.n, m = o.gmres_restart;
    const long ldm = n;
    GmresScratch G = gmres_scratch(S, m);
    const double *r = at<double>(S.work, S.L.R) + (long)c * n;
    std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m), sn(m), g(m + 1, 0.0), hb(2 * (m + 1) + 1);
    auto Hk = [&](int i, int j) -> double & { return H[(size_t)j * (m + 1) + i]; };
    g[0] = beta;
    *bad = false;
    MP_CUDA_TRY(launch_scale(n, r, beta, G.V, S.s));
    int k = 0;
    while (k < m) {
        double *vk = G.V + k * ldm, *w = G.V + (k + 1) * ldm, *zk = G.Z + k * ldm;
        // z_k = M v_k: the low-precision solve, v_k scaled by 2^ceil(log2 ||v_k||inf)
        MP_CUDA_TRY(cudaMemsetAsync(G.vnorm, 0, 3 * sizeof(double), S.s));
        MP_CUDA_TRY(launch_col_absmax(n, 1, vk, ldm, G.vnorm, &S.sb->gst, S.s));
        int e = lowp_solve<T>(S, vk, ldm, G.vnorm, 1);
        if (e) return e;
        MP_CUDA_TRY(launch_update<T>(n, 1, at<T>(S.work, S.L.Z), n, G.vnorm, zk, ldm, G.tn, 1, S.s));
        // w = A z_k in FP64
        MP_CUDA_TRY(cudaMemsetAsync(G.tn, 0, 2 * sizeof(double), S.s));
        if ((e = apply_A(S, 1, zk, ldm, nullptr, 0, w, ldm, G.tn, G.tn + 1, &S.sb->gst))) return e;
        // two passes of classical Gram-Schmidt against v_0..v_k, then ||w||_2^2
        MP_CUDA_TRY(launch_dots(n, k + 1, G.V, ldm, w, G.h1, S.s));
        MP_CUDA_TRY(launch_project(n, k + 1, G.V, ldm, G.h1, w, S.s));
        MP_CUDA_TRY(launch_dots(n, k + 1, G.V, ldm, w, G.h2, S.s));
        MP_CUDA_TRY(launch_project(n, k + 1, G.V, ldm, G.h2, w, S.s));
        MP_CUDA_TRY(launch_dots(n, 1, w, ldm, w, G.hh, S.s));
        MP_CUDA_TRY(cudaMemcpyAsync(hb.data(), G.h1, hb.size() * sizeof(double), cudaMemcpyDeviceToHost, S.s));
        MP_CUDA_TRY(cudaStreamSynchronize(S.s));
        for (int j = 0; j <= k; ++j) Hk(j, k) = hb[j] + hb[(m + 1) + j];
        const double hn = std::sqrt(hb[2 * (m + 1)]);
        Hk(k + 1, k) = hn;
        if (!std::isfinite(hn)) { *bad = true; break; }
        // earlier rotations on column k, then a new one zeroing H(k+1, k)
        for (int j = 0; j < k; ++j) {
            const double a = Hk(j, k), b = Hk(j + 1, k);
            Hk(j, k) = cs[j] * a + sn[j] * b;
            Hk(j + 1, k) = -sn[j] * a + cs[j] * b;
        }
        const double a = Hk(k, k), b = Hk(k + 1, k), den = std::hypot(a, b);
        cs[k] = den == 0.0 ? 1.0 : a / den;
        sn[k] = den == 0.0 ? 0.0 : b / den;
        Hk(k, k) = cs[k] * a + sn[k] * b;
        Hk(k + 1, k) = 0.0;
        g[k + 1] = -sn[k] * g[k];
        g[k] = cs[k] * g[k];
        ++k;
        // |g_{k}| is the residual norm of the small least-squares problem
        if (std::fabs(g[k]) <= std::max(o.gmres_tol * beta, floor) || hn == 0.0) break;
        MP_CUDA_TRY(launch_scale(n, w, hn, w, S.s));
    }
    *steps = k;
    if (*bad) return 0;
    // y = R_k^{-1} g_k (back substitution), then x_c += Z y
    std::vector<double> y(std::max(k, 1), 0.0);
    for (int i = k - 1; i >= 0; --i) {
        double t = g[i];
        for (int j = i + 1; j < k; ++j) t -= Hk(i, j) * y[j];
        y[i] = Hk(i, i) != 0.0 ? t / Hk(i, i) : 0.0;
        if (!std::isfinite(y[i])) *bad = true;
    }
    if (*bad || k == 0) return 0;
    MP_CUDA_TRY(cudaMemcpyAsync(G.y, y.data(), sizeof(double) * k, cudaMemcpyHostToDevice, S.s));
    MP_CUDA_TRY(launch_correct(n, k, G.Z, ldm, G.y, S.X + (long)c * S.ldx, &S.sb->znorm[c], S.s));
    return 0;
}

// Outer FP64 loop of GMRES-based refinement.  Starts from x_0 = M b unless
// from_x (then from the X the classical loop left).  Per column the
// acceptance rule of the classical loop (bwd <= tol at the FP64 floor), where
// the floor is also reached once ||r||_2 <= 4 sqrt(n) u64 ||A||inf ||x||inf
// (the residual is rounding noise); outer steps with no shrink of the
// correction and bwd > tol are a stall.
template <typename T>
int refine_gmres(Solve &S, const mp_opts &o, bool from_x, mp_stats *st, bool *conv, int *iters,
                 uint32_t *flags) {
    StatusBlock h;
    int e;
    *conv = false;
    *flags |= MP_FLAG_GMRES_USED;
    if (!from_x) {
        MP_CUDA_TRY(cudaMemsetAsync(S.sb->znorm, 0, sizeof(double) * kMaxRhs, S.s));
        if ((e = lowp_solve<T>(S, S.B, S.ldb, S.sb->bnorm, S.nrhs))) return e;
        MP_CUDA_TRY(launch_update<T>(S.n, S.nrhs, at<T>(S.work, S.L.Z), S.n, S.sb->bnorm, S.X, S.ldx,
                                     S.sb->znorm, 1, S.s));
        if (st) st->n_precond += 1;
    }
    double zprev[kMaxRhs] = {0};
    bool cdone[kMaxRhs] = {false};
    int it = 0;
    const double u64 = 1.1102230246251565e-16;
    for (;;) {
        if ((e = residual(S))) return e;
        for (int c = 0; c < S.nrhs; ++c)
            MP_CUDA_TRY(launch_dots(S.n, 1, at<double>(S.work, S.L.R) + (long)c * S.n, S.n,
                                    at<double>(S.work, S.L.R) + (long)c * S.n, &S.sb->rr[c], S.s));
        if ((e = read_status(S, h))) return e;
        double worst = 0.0;
        bool done = true, nonfinite = false, stalled = false, all_tol = true;
        for (int c = 0; c < S.nrhs; ++c) {
            const double b = bwd_of(h, c);
            const bool stagnant = it >= 2 && h.znorm[c] > o.stall_ratio * zprev[c];
            // a residual at the level at which it can be computed also marks
            // the floor: no GMRES cycle can determine a correction from it
            const bool r_floor = std::sqrt(h.rr[c]) <= 4.0 * std::sqrt((double)S.n) * u64 * h.st.anorm * h.xnorm[c];
            const bool at_floor =
                b == 0.0 || b <= 2.0 * u64 || h.znorm[c] <= 4.0 * u64 * h.xnorm[c] || stagnant || r_floor;
            cdone[c] = b <= o.tol && at_floor;
            if (!(b <= o.tol)) all_tol = false;
            if (!cdone[c]) done = false;
            if (!(b <= o.tol) && stagnant) stalled = true;
            if (!(b == b) || std::isinf(b)) nonfinite = true;
            worst = std::max(worst, std::isnan(b) ? INFINITY : b);
        }
        if (st) {
            if (st->nhist < 32) st->hist[st->nhist++] = worst;
            st->bwd_err = worst;
        }
        *flags |= h.st.flags & (MP_FLAG_TIMEOUT | MP_FLAG_NONFINITE_INPUT);
        if (h.st.flags & MP_FLAG_TIMEOUT) break;
        if (nonfinite) { *flags |= MP_FLAG_LOWP_BREAKDOWN; break; }
        if (done) { *conv = true; break; }
        if (stalled) { *flags |= MP_FLAG_STALLED; break; }
        if (it >= o.itermax) { *conv = all_tol; break; }
        std::memcpy(zprev, h.znorm, sizeof zprev);
        MP_CUDA_TRY(cudaMemsetAsync(S.sb->znorm, 0, sizeof(double) * kMaxRhs, S.s));
        bool bad = false;
        for (int c = 0; c < S.nrhs; ++c) {
            const double beta = std::sqrt(h.rr[c]);
            if (cdone[c] || !(beta > 0.0)) continue;
            int steps = 0;
            bool badc = false;
            const double floor = std::sqrt((double)S.n) * u64 * h.st.anorm * h.xnorm[c];
            if ((e = gmres_cycle<T>(S, o, c, beta, floor, &steps, &badc))) return e;
            if (st) st->n_precond += steps;
            bad = bad || badc;
        }
        if (bad) { *flags |= MP_FLAG_LOWP_BREAKDOWN; break; }
        ++it;
    }
    *iters = it;
    return 0;
}

int validate_opts(const mp_opts &o) {
    if (o.prec < MP_PREC_FP32 || o.prec > MP_PREC_FP64) return 1;
    if (o.itermax < 0 || !(o.tol > 0.0) || o.stall_ratio <= 0.0) return 1;
    if (o.refine < MP_REFINE_CLASSICAL || o.refine > MP_REFINE_AUTO) return 1;
    if (o.refine != MP_REFINE_CLASSICAL &&
        (o.gmres_restart < 1 || o.gmres_restart > 128 || !(o.gmres_tol > 0.0) || !(o.gmres_tol < 1.0)))
        return 1;
    return 0;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" size_t mp_gesv_workspace_bytes(int n, int nrhs, const mp_opts *opts) {
    mp_opts o;
    if (opts) o = *opts; else mp_default_opts(&o);
    if (n < 0 || nrhs < 0) return 0;
    return make_layout(n, nrhs, o, fp64_space_of(o)).total;
}

extern "C" int mp_gesv(int n, int nrhs, const double *dA, int lda, const double *dB, int ldb,
                       double *dX, int ldx, int32_t *dipiv, void *work, size_t work_bytes,
                       const mp_opts *opts, mp_stats *stats, void *stream) {
    return mp_gesv_impl(n, nrhs, dA, lda, dB, ldb, dX, ldx, dipiv, work, work_bytes, opts, stats, stream,
                        stats != nullptr);
}

// The driver behind mp_gesv (sym = false: PA = LU) and mp_posv (sym = true:
// A = L L^T from the lower triangle; no ipiv, arguments numbered without it).
int solve_impl(bool sym, int n, int nrhs, const double *dA, int lda, const double *dB, int ldb, double *dX,
               int ldx, int32_t *dipiv, void *work, size_t work_bytes, const mp_opts *opts, mp_stats *stats,
               void *stream, bool timing) {
    g_err[0] = 0;
    mp_opts o;
    if (opts) o = *opts; else mp_default_opts(&o);
    const int after = sym ? 1 : 0;  // arguments after ipiv shift down by one for posv
    if (n < 0) return mp_arg_fail(1, "n < 0");
    if (nrhs < 0 || nrhs > kMaxRhs) return mp_arg_fail(2, "nrhs must be in [0, 8]");
    if (n > 65536) return mp_arg_fail(1, "n > 65536 is not supported");
    if (n > 0 && !dA) return mp_arg_fail(3, "A is NULL");
    if (lda < std::max(1, n)) return mp_arg_fail(4, "lda < max(1, n)");
    if (n > 0 && nrhs > 0 && !dB) return mp_arg_fail(5, "B is NULL");
    if (ldb < std::max(1, n)) return mp_arg_fail(6, "ldb < max(1, n)");
    if (n > 0 && nrhs > 0 && !dX) return mp_arg_fail(7, "X is NULL");
    if (ldx < std::max(1, n)) return mp_arg_fail(8, "ldx < max(1, n)");
    if (!sym && n > 0 && !dipiv) return mp_arg_fail(9, "ipiv is NULL");
    if (validate_opts(o)) return mp_arg_fail(12 - after, "invalid options");
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
    }
    if (n == 0 || nrhs == 0) return 0;
    const bool plain64 = o.prec == MP_PREC_FP64;  // the plain FP64 solve, no low precision
    const bool fb = o.allow_fallback != 0 && !plain64;
    Layout L = make_layout(n, nrhs, o, fp64_space_of(o), sym);
    if (!work) return mp_arg_fail(10 - after, "workspace is NULL");
    if (work_bytes < L.total) return mp_arg_fail(11 - after, "workspace too small");

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Solve S{n, nrhs, dA, lda, dB, ldb, dX, ldx, work, L, s, at<StatusBlock>(work, L.status), 0, sym};
    cudaEvent_t ev[5] = {};
    if (timing)
        for (auto &e : ev) MP_CUDA_TRY(cudaEventCreate(&e));
    auto mark = [&](int i) { if (timing) cudaEventRecord(ev[i], s); };
    auto convert = [&](auto *W) -> cudaError_t {
        using T = std::remove_pointer_t<decltype(W)>;
        return sym ? launch_convert_lower<T>(n, dA, lda, W, L.ldw, at<double>(work, L.rowsum), &S.sb->st, s)
                   : launch_convert_transpose<T>(n, dA, lda, W, L.ldw, at<double>(work, L.rowsum), &S.sb->st, s);
    };

    mark(0);
    MP_CUDA_TRY(cudaMemsetAsync(S.sb, 0, sizeof(StatusBlock), s));
    MP_CUDA_TRY(cudaMemsetAsync(at<double>(work, L.rowsum), 0, sizeof(double) * n, s));
    if (reset_sync(S)) return -1000;
    if (plain64)
        MP_CUDA_TRY(convert(at<double>(work, L.W)));
    else
        MP_CUDA_TRY(convert(at<float>(work, L.W)));
    MP_CUDA_TRY(launch_max_reduce(n, at<double>(work, L.rowsum), &S.sb->st.anorm, s));
    MP_CUDA_TRY(launch_col_absmax(n, nrhs, dB, ldb, S.sb->bnorm, &S.sb->st, s));
    mark(1);

    uint32_t flags = 0;
    int info = 0, iters = 0, e;
    bool conv = false;
    uint32_t fflags = 0;
    if (plain64) {
        // The plain double-precision solver the paper measures its speedups
        // against (Section 3: DGETRF + DGETRS, DPOTRF + DPOTRS): FP64 factors,
        // x_0 from them, and the same acceptance test (corrections, if any,
        // with the FP64 factors).  The answer is FP64 throughout, so no
        // fallback flag.
        int ret = 0;
        if ((e = factor<double>(S, MP_PREC_FP32, std::min(L.nb, 256), &info, &fflags))) return e;
        mark(2);
        flags |= fflags & MP_FLAG_NONFINITE_INPUT;
        if (info > 0) {
            ret = info;
        } else if (!(flags & MP_FLAG_NONFINITE_INPUT)) {
            if ((e = refine<double>(S, o, o.itermax, false, stats, &conv, &iters, &flags))) return e;
            if (!conv) flags |= MP_FLAG_NOT_CONVERGED;
        }
        mark(3);
        if (!sym)
            MP_CUDA_TRY(cudaMemcpyAsync(dipiv, at<int32_t>(work, L.ipiv), sizeof(int32_t) * n,
                                        cudaMemcpyDeviceToDevice, s));
        {
            const int kind = ret != 0 ? kNoFactors : sym ? kCholF64 : kLuF64;
            MP_CUDA_TRY(cudaMemcpyAsync(&S.sb->factor_kind, &kind, sizeof(int), cudaMemcpyHostToDevice, s));
        }
        mark(4);
        MP_CUDA_TRY(cudaStreamSynchronize(s));
        if (stats) {
            stats->iter = iters;
            stats->flags = flags;
            stats->info = info;
            if (timing) {
                cudaEventElapsedTime(&stats->ms_convert, ev[0], ev[1]);
                cudaEventElapsedTime(&stats->ms_factor, ev[1], ev[2]);
                cudaEventElapsedTime(&stats->ms_refine, ev[2], ev[3]);
            }
        }
        if (timing)
            for (auto &x : ev) cudaEventDestroy(x);
        return ret;
    }
    if ((e = factor<float>(S, o.prec, L.nb, &info, &fflags))) return e;
    mark(2);
    flags |= fflags & (MP_FLAG_LOWP_BREAKDOWN | MP_FLAG_NONFINITE_INPUT);
    if (!(flags & (MP_FLAG_LOWP_BREAKDOWN | MP_FLAG_NONFINITE_INPUT))) {
        if (o.refine == MP_REFINE_GMRES) {
            if ((e = refine_gmres<float>(S, o, false, stats, &conv, &iters, &flags))) return e;
        } else {
            if ((e = refine<float>(S, o, o.itermax, true, stats, &conv, &iters, &flags))) return e;
            // AUTO: a classical loop that stalled or ran out of corrections
            // continues with GMRES on the same factors (Section 2.2)
            const uint32_t hard = MP_FLAG_LOWP_BREAKDOWN | MP_FLAG_NONFINITE_INPUT | MP_FLAG_TIMEOUT;
            if (!conv && o.refine == MP_REFINE_AUTO && !(flags & hard)) {
                int itg = 0;
                if ((e = refine_gmres<float>(S, o, true, stats, &conv, &itg, &flags))) return e;
                iters += itg;
            }
        }
    }
    if (stats) stats->info = info;
    mark(3);
    int ret = 0;
    if (!conv && fb && !(flags & MP_FLAG_NONFINITE_INPUT)) {
        // Section 4: resort to the double-precision solver (FP64 LU or
        // Cholesky on the GPU, the same kernels instantiated for FP64)
        MP_CUDA_TRY(cudaMemsetAsync(&S.sb->st.zero_pivot, 0, sizeof(int), s));
        MP_CUDA_TRY(cudaMemsetAsync(&S.sb->st.flags, 0, sizeof(uint32_t), s));
        if (reset_sync(S)) return -1000;
        MP_CUDA_TRY(convert(at<double>(work, L.W)));
        int info64 = 0;
        uint32_t f64 = 0;
        if ((e = factor<double>(S, MP_PREC_FP32, std::min(L.nb, 256), &info64, &f64))) return e;
        flags |= MP_FLAG_FALLBACK;
        if (info64 > 0) {
            ret = info64;
        } else {
            bool conv64 = false;
            int it64 = 0;
            uint32_t fl64 = 0;
            if ((e = refine<double>(S, o, 5, false, nullptr, &conv64, &it64, &fl64))) return e;
            flags |= fl64 & MP_FLAG_TIMEOUT;
            StatusBlock h;
            if ((e = read_status(S, h))) return e;
            double worst = 0.0;
            for (int c = 0; c < nrhs; ++c) worst = std::max(worst, bwd_of(h, c));
            if (stats) stats->bwd_err = worst;
        }
        iters = -1;
    } else if (!conv) {
        flags |= MP_FLAG_NOT_CONVERGED;
    }
    if (!sym)
        MP_CUDA_TRY(cudaMemcpyAsync(dipiv, at<int32_t>(work, L.ipiv), sizeof(int32_t) * n,
                                    cudaMemcpyDeviceToDevice, s));
    {
        // the factors now in the workspace, for mp_gesv_adjoint
        const bool f64 = (flags & MP_FLAG_FALLBACK) != 0;
        const int kind = ret != 0 ? kNoFactors : sym ? (f64 ? kCholF64 : kCholF32) : (f64 ? kLuF64 : kLuF32);
        MP_CUDA_TRY(cudaMemcpyAsync(&S.sb->factor_kind, &kind, sizeof(int), cudaMemcpyHostToDevice, s));
    }
    mark(4);
    MP_CUDA_TRY(cudaStreamSynchronize(s));
    if (stats) {
        stats->iter = iters;
        stats->flags = flags;
        if (timing && stats) {
            cudaEventElapsedTime(&stats->ms_convert, ev[0], ev[1]);
            cudaEventElapsedTime(&stats->ms_factor, ev[1], ev[2]);
            cudaEventElapsedTime(&stats->ms_refine, ev[2], ev[3]);
            cudaEventElapsedTime(&stats->ms_fallback, ev[3], ev[4]);
        }
    }
    if (timing)
        for (auto &ev_ : ev) cudaEventDestroy(ev_);
    return ret;
}

int mp_gesv_impl(int n, int nrhs, const double *dA, int lda, const double *dB, int ldb, double *dX,
                 int ldx, int32_t *dipiv, void *work, size_t work_bytes, const mp_opts *opts,
                 mp_stats *stats, void *stream, bool timing) {
    return solve_impl(false, n, nrhs, dA, lda, dB, ldb, dX, ldx, dipiv, work, work_bytes, opts, stats, stream,
                      timing);
}

extern "C" size_t mp_posv_workspace_bytes(int n, int nrhs, const mp_opts *opts) {
    mp_opts o;
    if (opts) o = *opts; else mp_default_opts(&o);
    if (n < 0 || nrhs < 0) return 0;
    return make_layout(n, nrhs, o, fp64_space_of(o), true).total;
}

extern "C" int mp_posv(int n, int nrhs, const double *dA, int lda, const double *dB, int ldb, double *dX,
                       int ldx, void *work, size_t work_bytes, const mp_opts *opts, mp_stats *stats,
                       void *stream) {
    return solve_impl(true, n, nrhs, dA, lda, dB, ldb, dX, ldx, nullptr, work, work_bytes, opts, stats, stream,
                      stats != nullptr);
}

// ---------------------------------------------------------------------------
// Adjoint of the solve (the reverse-mode derivative of X = A^{-1} B; not in
// the paper): Bbar = A^{-T} G by transposed solves with the factors the
// forward call left in its workspace, refined in FP64 against A^T exactly as
// Algorithm 1 refines against A, then Abar = -Bbar X^T.
// ---------------------------------------------------------------------------
namespace {
struct AdjLayout {
    size_t Wt, Linv, Uinv, tmp, total;
};
AdjLayout adj_layout(int n, bool fp64) {
    AdjLayout L{};
    const size_t el = fp64 ? sizeof(double) : sizeof(float);
    size_t off = 0;
    L.Wt = carve(off, (size_t)n * (size_t)mp_factor_ld(n) * el);
    const size_t inv = std::max(trsv_inverse_bytes<float>(n), fp64 ? trsv_inverse_bytes<double>(n) : 0);
    L.Linv = carve(off, inv);
    L.Uinv = carve(off, inv);
    L.tmp = carve(off, std::max(trsv_tmp_bytes<float>(n), fp64 ? trsv_tmp_bytes<double>(n) : 0));
    L.total = align_up(off, 256);
    return L;
}

template <typename T>
int adjoint_solve(Solve &S, const mp_opts &o, void *adj, const AdjLayout &AL, mp_stats *st, bool *conv, int *iters,
                  uint32_t *flags) {
    if (!S.sym) {
        // A^T = U^T L^T P: W^T has U^T in its lower triangle, L^T (unit) in its upper
        T *W = at<T>(S.work, S.L.W);
        T *Wt = at<T>(adj, AL.Wt);
        MP_CUDA_TRY(launch_transpose<T>(S.n, W, S.L.ldw, Wt, S.L.ldw, S.s));
        MP_CUDA_TRY(launch_build_inverses<T>(S.n, Wt, S.L.ldw, at<T>(adj, AL.Linv), at<T>(adj, AL.Uinv),
                                             at<T>(adj, AL.tmp), S.s, false, true));
        S.trans = true;
        S.tW = Wt;
        S.tLinv = at<T>(adj, AL.Linv);
        S.tUinv = at<T>(adj, AL.Uinv);
    }
    // (for Cholesky A^T = A: the forward factors serve unchanged)
    return refine<T>(S, o, o.itermax, true, st, conv, iters, flags);
}
}  // namespace

extern "C" size_t mp_gesv_adjoint_workspace_bytes(int n, const mp_opts *opts) {
    mp_opts o;
    if (opts) o = *opts; else mp_default_opts(&o);
    if (n < 0) return 0;
    return adj_layout(n, fp64_space_of(o)).total;
}

extern "C" int mp_gesv_adjoint(int n, int nrhs, const double *dA, int lda, const double *dX, int ldx,
                               const double *dG, int ldg, double *dBbar, int ldbb, double *dAbar, int ldab,
                               void *work, size_t work_bytes, void *adj_work, size_t adj_bytes,
                               const mp_opts *opts, mp_stats *stats, void *stream) {
    g_err[0] = 0;
    mp_opts o;
    if (opts) o = *opts; else mp_default_opts(&o);
    if (n < 0) return mp_arg_fail(1, "n < 0");
    if (nrhs < 0 || nrhs > kMaxRhs) return mp_arg_fail(2, "nrhs must be in [0, 8]");
    if (n > 65536) return mp_arg_fail(1, "n > 65536 is not supported");
    if (n > 0 && !dA) return mp_arg_fail(3, "A is NULL");
    if (lda < std::max(1, n)) return mp_arg_fail(4, "lda < max(1, n)");
    if (n > 0 && nrhs > 0 && !dX) return mp_arg_fail(5, "X is NULL");
    if (ldx < std::max(1, n)) return mp_arg_fail(6, "ldx < max(1, n)");
    if (n > 0 && nrhs > 0 && !dG) return mp_arg_fail(7, "G is NULL");
    if (ldg < std::max(1, n)) return mp_arg_fail(8, "ldg < max(1, n)");
    if (n > 0 && nrhs > 0 && !dBbar) return mp_arg_fail(9, "Bbar is NULL");
    if (ldbb < std::max(1, n)) return mp_arg_fail(10, "ldbb < max(1, n)");
    if (ldab < std::max(1, n)) return mp_arg_fail(12, "ldab < max(1, n)");
    if (validate_opts(o)) return mp_arg_fail(17, "invalid options");
    o.refine = MP_REFINE_CLASSICAL;  // the transposed system is refined by Algorithm 1
    if (stats) std::memset(stats, 0, sizeof(*stats));
    if (n == 0) return 0;
    if (!work) return mp_arg_fail(13, "workspace is NULL");
    if (work_bytes < sizeof(StatusBlock)) return mp_arg_fail(14, "workspace too small");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    StatusBlock *sb = static_cast<StatusBlock *>(work);  // first region of every solve layout
    int kind = 0;
    MP_CUDA_TRY(cudaMemcpyAsync(&kind, &sb->factor_kind, sizeof(int), cudaMemcpyDeviceToHost, s));
    MP_CUDA_TRY(cudaStreamSynchronize(s));
    if (kind == kNoFactors || kind > kCholF64)
        return mp_arg_fail(13, "workspace holds no factors of a finished mp_gesv / mp_posv");
    const bool sym = kind == kCholF32 || kind == kCholF64;
    const bool f64 = kind == kLuF64 || kind == kCholF64;
    Layout L = make_layout(n, std::max(nrhs, 1), o, fp64_space_of(o), sym);
    if (work_bytes < L.total) return mp_arg_fail(14, "workspace too small for (n, nrhs, opts)");
    if (f64 && !fp64_space_of(o))
        return mp_arg_fail(17, "FP64 factors need allow_fallback = 1 (or prec FP64) in opts");
    AdjLayout AL = adj_layout(n, fp64_space_of(o));
    if (!sym && !adj_work) return mp_arg_fail(15, "adjoint workspace is NULL");
    if (!sym && adj_bytes < AL.total) return mp_arg_fail(16, "adjoint workspace too small");
    if (nrhs == 0) return 0;
    if (!dAbar) return mp_arg_fail(11, "Abar is NULL");

    Solve S{n, nrhs, dA, lda, dG, ldg, dBbar, ldbb, work, L, s, sb, 0, sym};
    // status words of this solve (the factor record stays)
    MP_CUDA_TRY(cudaMemsetAsync(&sb->st.flags, 0, sizeof(uint32_t), s));
    MP_CUDA_TRY(cudaMemsetAsync(sb->bnorm, 0, sizeof(double) * kMaxRhs, s));
    if (reset_sync(S)) return -1000;
    MP_CUDA_TRY(launch_col_absmax(n, nrhs, dG, ldg, sb->bnorm, &sb->st, s));
    bool conv = false;
    int iters = 0, e;
    uint32_t flags = 0;
    if (f64) e = adjoint_solve<double>(S, o, adj_work, AL, stats, &conv, &iters, &flags);
    else e = adjoint_solve<float>(S, o, adj_work, AL, stats, &conv, &iters, &flags);
    if (e) return e;
    if (!conv) flags |= MP_FLAG_NOT_CONVERGED;
    if (f64 && o.prec != MP_PREC_FP64) flags |= MP_FLAG_FALLBACK;
    MP_CUDA_TRY(launch_outer_neg(n, nrhs, dBbar, ldbb, dX, ldx, dAbar, ldab, s));
    MP_CUDA_TRY(cudaStreamSynchronize(s));
    if (stats) {
        stats->iter = iters;
        stats->flags = flags;
    }
    return 0;
}

extern "C" size_t mp_gesv_host_workspace_bytes(int n, int nrhs, const mp_opts *opts) {
    if (n < 0 || nrhs < 0) return 0;
    size_t off = 0;
    carve(off, sizeof(double) * (size_t)n * n);
    carve(off, sizeof(double) * (size_t)n * std::max(nrhs, 1));
    carve(off, sizeof(double) * (size_t)n * std::max(nrhs, 1));
    carve(off, sizeof(int32_t) * (size_t)std::max(n, 1));
    off = align_up(off, 256);
    return off + mp_gesv_workspace_bytes(n, nrhs, opts);
}

extern "C" int mp_gesv_host(int n, int nrhs, const double *hA, int lda, const double *hB, int ldb,
                            double *hX, int ldx, int32_t *hipiv, void *work, size_t work_bytes,
                            const mp_opts *opts, mp_stats *stats, void *stream) {
    g_err[0] = 0;
    if (n < 0) return mp_arg_fail(1, "n < 0");
    if (nrhs < 0 || nrhs > kMaxRhs) return mp_arg_fail(2, "nrhs must be in [0, 8]");
    if (n > 0 && !hA) return mp_arg_fail(3, "A is NULL");
    if (lda < std::max(1, n)) return mp_arg_fail(4, "lda < max(1, n)");
    if (n > 0 && nrhs > 0 && !hB) return mp_arg_fail(5, "B is NULL");
    if (ldb < std::max(1, n)) return mp_arg_fail(6, "ldb < max(1, n)");
    if (n > 0 && nrhs > 0 && !hX) return mp_arg_fail(7, "X is NULL");
    if (ldx < std::max(1, n)) return mp_arg_fail(8, "ldx < max(1, n)");
    if (n > 0 && !hipiv) return mp_arg_fail(9, "ipiv is NULL");
    if (n == 0 || nrhs == 0) return 0;
    if (!work) return mp_arg_fail(10, "workspace is NULL");
    if (work_bytes < mp_gesv_host_workspace_bytes(n, nrhs, opts)) return mp_arg_fail(11, "workspace too small");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    size_t off = 0;
    double *dA = at<double>(work, carve(off, sizeof(double) * (size_t)n * n));
    double *dB = at<double>(work, carve(off, sizeof(double) * (size_t)n * nrhs));
    double *dX = at<double>(work, carve(off, sizeof(double) * (size_t)n * nrhs));
    int32_t *dp = at<int32_t>(work, carve(off, sizeof(int32_t) * (size_t)n));
    off = align_up(off, 256);
    MP_CUDA_TRY(cudaMemcpy2DAsync(dA, sizeof(double) * n, hA, sizeof(double) * lda, sizeof(double) * n, n,
                                  cudaMemcpyHostToDevice, s));
    MP_CUDA_TRY(cudaMemcpy2DAsync(dB, sizeof(double) * n, hB, sizeof(double) * ldb, sizeof(double) * n,
                                  nrhs, cudaMemcpyHostToDevice, s));
    int r = mp_gesv(n, nrhs, dA, n, dB, n, dX, n, dp, static_cast<char *>(work) + off, work_bytes - off,
                    opts, stats, stream);
    if (r < 0 && r > -1000) return r;  // argument errors are not expected here
    MP_CUDA_TRY(cudaMemcpy2DAsync(hX, sizeof(double) * ldx, dX, sizeof(double) * n, sizeof(double) * n,
                                  nrhs, cudaMemcpyDeviceToHost, s));
    MP_CUDA_TRY(cudaMemcpyAsync(hipiv, dp, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
    MP_CUDA_TRY(cudaStreamSynchronize(s));
    return r;
}

// ---------------------------------------------------------------------------
// step entry points
// ---------------------------------------------------------------------------
namespace {
struct StepLayout {
    size_t status, rowsum, perm, pairs, npairs, map, Linv, Uinv, invtmp, acc, bar, Y, Z, part, tc, linv, total;
    int nblk, ksplit;
};
StepLayout step_layout(int n, int nrhs, int nb, int prec) {
    StepLayout L{};
    L.nblk = (n + 127) / 128;
    L.ksplit = residual_ksplit(std::max(n, 1), std::max(nrhs, 1));
    const int rhs = std::max(nrhs, 1);
    size_t off = 0;
    L.status = carve(off, sizeof(StatusBlock));
    L.rowsum = carve(off, sizeof(double) * (size_t)n);
    L.perm = carve(off, sizeof(int) * (size_t)n);
    L.pairs = carve(off, sizeof(int2) * ((size_t)2 * (size_t)std::max(n, nb) + 128));
    L.npairs = carve(off, sizeof(int) * 32);  // [0], [1]: two leaves' move counts, [2]: max |U12|, [4..20): tickets
    L.map = carve(off, sizeof(int) * (size_t)n);
    L.Linv = carve(off, trsv_inverse_bytes<float>(n));
    L.Uinv = carve(off, trsv_inverse_bytes<float>(n));
    L.invtmp = carve(off, trsv_tmp_bytes<float>(n));
    L.acc = carve(off, sizeof(float) * (size_t)n * rhs);
    L.bar = carve(off, trsv_sync_bytes<float>(n));
    L.Y = carve(off, sizeof(float) * (size_t)n * rhs);
    L.Z = carve(off, sizeof(float) * (size_t)n * rhs);
    L.part = carve(off, sizeof(double) * (size_t)L.ksplit * n * rhs);
    L.tc = carve(off, prec == MP_PREC_FP32 ? 0
                                           : std::max(tc_workspace_bytes(n, nb, prec),
                                                      tc_workspace_bytes(n, nb, MP_PREC_FP16X3)));
    L.linv = carve(off, 3 * 1024 * sizeof(double));
    L.total = align_up(off, 256);
    return L;
}
}  // namespace

extern "C" size_t mp_getrf_workspace_bytes(int n, const mp_opts *opts) {
    mp_opts o;
    if (opts) o = *opts; else mp_default_opts(&o);
    if (n < 0) return 0;
    return step_layout(n, 1, outer_nb(n, o), o.prec).total;
}
extern "C" size_t mp_getrs_workspace_bytes(int n, int nrhs) {
    if (n < 0 || nrhs < 0) return 0;
    return step_layout(n, nrhs, 32, MP_PREC_FP32).total;
}
extern "C" size_t mp_residual_workspace_bytes(int n, int nrhs) {
    if (n < 0 || nrhs < 0) return 0;
    return step_layout(n, nrhs, 32, MP_PREC_FP32).total;
}

extern "C" int mp_convert(int n, const double *dA, int lda, float *dW, int ldw, double *d_anorm,
                          uint32_t *d_flags, void *work, size_t work_bytes, void *stream) {
    g_err[0] = 0;
    if (n < 0) return mp_arg_fail(1, "n < 0");
    if (n > 0 && !dA) return mp_arg_fail(2, "A is NULL");
    if (lda < std::max(1, n)) return mp_arg_fail(3, "lda < max(1, n)");
    if (n > 0 && !dW) return mp_arg_fail(4, "W is NULL");
    if (ldw < std::max(1, n)) return mp_arg_fail(5, "ldw < max(1, n)");
    if (!d_anorm) return mp_arg_fail(6, "anorm is NULL");
    if (!d_flags) return mp_arg_fail(7, "flags is NULL");
    StepLayout L = step_layout(n, 1, 32, MP_PREC_FP32);
    if (!work) return mp_arg_fail(8, "workspace is NULL");
    if (work_bytes < L.total) return mp_arg_fail(9, "workspace too small");
    if (n == 0) return 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    StatusBlock *sb = at<StatusBlock>(work, L.status);
    MP_CUDA_TRY(cudaMemsetAsync(sb, 0, sizeof(StatusBlock), s));
    MP_CUDA_TRY(cudaMemsetAsync(at<double>(work, L.rowsum), 0, sizeof(double) * n, s));
    MP_CUDA_TRY(launch_convert_transpose<float>(n, dA, lda, dW, ldw, at<double>(work, L.rowsum), &sb->st, s));
    MP_CUDA_TRY(launch_max_reduce(n, at<double>(work, L.rowsum), d_anorm, s));
    MP_CUDA_TRY(cudaMemcpyAsync(d_flags, &sb->st.flags, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    return 0;
}

extern "C" int mp_getrf_lowp(int n, float *dW, int ldw, int32_t *dipiv, const mp_opts *opts, void *work,
                             size_t work_bytes, int *info, uint32_t *flags, void *stream) {
    g_err[0] = 0;
    mp_opts o;
    if (opts) o = *opts; else mp_default_opts(&o);
    if (n < 0 || n > 65536) return mp_arg_fail(1, "n out of range [0, 65536]");
    if (n > 0 && !dW) return mp_arg_fail(2, "W is NULL");
    if (ldw < mp_factor_ld(n) || ldw % 32) return mp_arg_fail(3, "ldw must be a multiple of 32 >= n");
    if (n > 0 && !dipiv) return mp_arg_fail(4, "ipiv is NULL");
    if (validate_opts(o) || o.prec == MP_PREC_FP64) return mp_arg_fail(5, "invalid options");
    const int nb = outer_nb(n, o);
    StepLayout L = step_layout(n, 1, nb, o.prec);
    if (!work) return mp_arg_fail(6, "workspace is NULL");
    if (work_bytes < L.total) return mp_arg_fail(7, "workspace too small");
    if (info) *info = 0;
    if (flags) *flags = 0;
    if (n == 0) return 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    StatusBlock *sb = at<StatusBlock>(work, L.status);
    MP_CUDA_TRY(cudaMemsetAsync(sb, 0, sizeof(StatusBlock), s));
    MP_CUDA_TRY(launch_iota(at<int>(work, L.perm), n, s));
    MP_CUDA_TRY(launch_iota(at<int>(work, L.map), n, s));
    FactorCtx<float> c{dW, (long)ldw, n, dipiv, at<int>(work, L.perm), at<int2>(work, L.pairs),
                       at<int>(work, L.npairs), at<int>(work, L.map), &sb->st, s, o.prec, at<void>(work, L.tc),
                       at<float>(work, L.linv)};
    MP_CUDA_TRY(getrf_blocked<float>(c, nb));
    StatusBlock h;
    MP_CUDA_TRY(cudaMemcpyAsync(&h, sb, sizeof h, cudaMemcpyDeviceToHost, s));
    MP_CUDA_TRY(cudaStreamSynchronize(s));
    if (info) *info = h.st.zero_pivot;
    if (flags) *flags = h.st.flags;
    return 0;
}

extern "C" int mp_potrf_lowp(int n, float *dW, int ldw, const mp_opts *opts, void *work, size_t work_bytes,
                             int *info, uint32_t *flags, void *stream) {
    g_err[0] = 0;
    mp_opts o;
    if (opts) o = *opts; else mp_default_opts(&o);
    if (n < 0 || n > 65536) return mp_arg_fail(1, "n out of range [0, 65536]");
    if (n > 0 && !dW) return mp_arg_fail(2, "W is NULL");
    if (ldw < mp_factor_ld(n) || ldw % 32) return mp_arg_fail(3, "ldw must be a multiple of 32 >= n");
    if (validate_opts(o) || o.prec == MP_PREC_FP64) return mp_arg_fail(4, "invalid options");
    const int nb = outer_nb(n, o);
    StepLayout L = step_layout(n, 1, nb, o.prec);
    if (!work) return mp_arg_fail(5, "workspace is NULL");
    if (work_bytes < L.total) return mp_arg_fail(6, "workspace too small");
    if (info) *info = 0;
    if (flags) *flags = 0;
    if (n == 0) return 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    StatusBlock *sb = at<StatusBlock>(work, L.status);
    MP_CUDA_TRY(cudaMemsetAsync(sb, 0, sizeof(StatusBlock), s));
    FactorCtx<float> c{dW, (long)ldw, n, nullptr, at<int>(work, L.perm), at<int2>(work, L.pairs),
                       at<int>(work, L.npairs), at<int>(work, L.map), &sb->st, s, o.prec, at<void>(work, L.tc)};
    MP_CUDA_TRY(potrf_blocked<float>(c, nb));
    StatusBlock h;
    MP_CUDA_TRY(cudaMemcpyAsync(&h, sb, sizeof h, cudaMemcpyDeviceToHost, s));
    MP_CUDA_TRY(cudaStreamSynchronize(s));
    if (info) *info = h.st.zero_pivot;
    if (flags) *flags = h.st.flags;
    return 0;
}

extern "C" int mp_getrs_lowp(int n, int nrhs, const float *dW, int ldw, const int32_t *dipiv,
                             const double *dR, int ldr, double *dZ, int ldz, void *work,
                             size_t work_bytes, void *stream) {
    g_err[0] = 0;
    if (n < 0) return mp_arg_fail(1, "n < 0");
    if (nrhs < 0 || nrhs > kMaxRhs) return mp_arg_fail(2, "nrhs must be in [0, 8]");
    if (n > 0 && !dW) return mp_arg_fail(3, "W is NULL");
    if (ldw < std::max(1, n) || ldw % 4) return mp_arg_fail(4, "ldw must be >= n and a multiple of 4");
    if (n > 0 && !dipiv) return mp_arg_fail(5, "ipiv is NULL");
    if (n > 0 && nrhs > 0 && !dR) return mp_arg_fail(6, "R is NULL");
    if (ldr < std::max(1, n)) return mp_arg_fail(7, "ldr < max(1, n)");
    if (n > 0 && nrhs > 0 && !dZ) return mp_arg_fail(8, "Z is NULL");
    if (ldz < std::max(1, n)) return mp_arg_fail(9, "ldz < max(1, n)");
    StepLayout L = step_layout(n, nrhs, 32, MP_PREC_FP32);
    if (!work) return mp_arg_fail(10, "workspace is NULL");
    if (work_bytes < L.total) return mp_arg_fail(11, "workspace too small");
    if (n == 0 || nrhs == 0) return 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    StatusBlock *sb = at<StatusBlock>(work, L.status);
    MP_CUDA_TRY(cudaMemsetAsync(sb, 0, sizeof(StatusBlock), s));
    MP_CUDA_TRY(cudaMemsetAsync(at<unsigned>(work, L.bar), 0, sizeof(unsigned) * 4, s));
    // row permutation from the pivots: compose all n swaps, apply to identity
    int *perm = at<int>(work, L.perm);
    MP_CUDA_TRY(launch_iota(perm, n, s));
    MP_CUDA_TRY(launch_iota(at<int>(work, L.map), n, s));
    const int chunk = 4096;  // compose in chunks (bounded shared memory for the pivot copy)
    for (int k = 0; k < n; k += chunk) {
        const int k2 = std::min(n, k + chunk);
        MP_CUDA_TRY(launch_compose_swaps(dipiv, k, k2, n, at<int2>(work, L.pairs), at<int>(work, L.npairs),
                                         at<int>(work, L.map), s));
        MP_CUDA_TRY(launch_apply_moves_vec(perm, at<int2>(work, L.pairs), at<int>(work, L.npairs),
                                           2 * (k2 - k), s));
    }
    MP_CUDA_TRY(launch_build_inverses<float>(n, dW, ldw, at<float>(work, L.Linv), at<float>(work, L.Uinv),
                                             at<float>(work, L.invtmp), s));
    MP_CUDA_TRY(launch_col_absmax(n, nrhs, dR, ldr, sb->rnorm, &sb->st, s));
    MP_CUDA_TRY(launch_trsv_lower<float>(n, nrhs, dW, ldw, at<float>(work, L.Linv), dR, ldr, perm, sb->rnorm,
                                         at<float>(work, L.Y), n, at<float>(work, L.acc),
                                         at<unsigned>(work, L.bar), &sb->st, s));
    MP_CUDA_TRY(launch_trsv_upper<float>(n, nrhs, dW, ldw, at<float>(work, L.Uinv), at<float>(work, L.Y), n,
                                         at<float>(work, L.Z), n, at<float>(work, L.acc),
                                         at<unsigned>(work, L.bar), &sb->st, s));
    MP_CUDA_TRY(launch_update<float>(n, nrhs, at<float>(work, L.Z), n, sb->rnorm, dZ, ldz, sb->znorm, 1, s));
    StatusBlock h;
    MP_CUDA_TRY(cudaMemcpyAsync(&h, sb, sizeof h, cudaMemcpyDeviceToHost, s));
    MP_CUDA_TRY(cudaStreamSynchronize(s));
    if (h.st.flags & MP_FLAG_TIMEOUT) {
        mp_set_error("triangular solve: a bounded wait gave up");
        return -1000 - (int)cudaErrorLaunchTimeout;
    }
    return 0;
}

extern "C" int mp_residual(int n, int nrhs, const double *dA, int lda, const double *dX, int ldx,
                           const double *dB, int ldb, double *dR, int ldr, void *work, size_t work_bytes,
                           void *stream) {
    g_err[0] = 0;
    if (n < 0) return mp_arg_fail(1, "n < 0");
    if (nrhs < 0 || nrhs > kMaxRhs) return mp_arg_fail(2, "nrhs must be in [0, 8]");
    if (n > 0 && !dA) return mp_arg_fail(3, "A is NULL");
    if (lda < std::max(1, n)) return mp_arg_fail(4, "lda < max(1, n)");
    if (n > 0 && nrhs > 0 && !dX) return mp_arg_fail(5, "X is NULL");
    if (ldx < std::max(1, n)) return mp_arg_fail(6, "ldx < max(1, n)");
    if (n > 0 && nrhs > 0 && !dB) return mp_arg_fail(7, "B is NULL");
    if (ldb < std::max(1, n)) return mp_arg_fail(8, "ldb < max(1, n)");
    if (n > 0 && nrhs > 0 && !dR) return mp_arg_fail(9, "R is NULL");
    if (ldr < std::max(1, n)) return mp_arg_fail(10, "ldr < max(1, n)");
    StepLayout L = step_layout(n, nrhs, 32, MP_PREC_FP32);
    if (!work) return mp_arg_fail(11, "workspace is NULL");
    if (work_bytes < L.total) return mp_arg_fail(12, "workspace too small");
    if (n == 0 || nrhs == 0) return 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    StatusBlock *sb = at<StatusBlock>(work, L.status);
    MP_CUDA_TRY(cudaMemsetAsync(sb, 0, sizeof(StatusBlock), s));
    MP_CUDA_TRY(launch_residual_partial(n, nrhs, dA, lda, dX, ldx, at<double>(work, L.part), L.ksplit, s));
    MP_CUDA_TRY(launch_residual_finalize(n, nrhs, at<double>(work, L.part), L.ksplit, dB, ldb, dX, ldx, dR,
                                         ldr, sb->rnorm, sb->xnorm, &sb->st, s));
    return 0;
}

extern "C" size_t mp_lowp_gemm_workspace_bytes(int M, int N, int K, int prec) {
    if (M < 0 || N < 0 || K < 0) return 0;
    size_t off = 0;
    carve(off, sizeof(StatusBlock));
    carve(off, tc_workspace_bytes(std::max(M, N), K, prec));
    return align_up(off, 256);
}

extern "C" int mp_lowp_gemm_update(int prec, int M, int N, int K, const float *dL, int ldl, const float *dU,
                                   int ldu, float *dC, int ldc, void *work, size_t work_bytes, void *stream) {
    g_err[0] = 0;
    if (prec != MP_PREC_FP32 && prec != MP_PREC_BF16 && prec != MP_PREC_FP16 && prec != MP_PREC_FP16X3 &&
        prec != MP_PREC_E4M3)
        return mp_arg_fail(1, "prec must be FP32, FP16X3, BF16, FP16 or E4M3");
    if (M < 0) return mp_arg_fail(2, "M < 0");
    if (N < 0) return mp_arg_fail(3, "N < 0");
    if (K < 0) return mp_arg_fail(4, "K < 0");
    if (M > 0 && K > 0 && !dL) return mp_arg_fail(5, "L is NULL");
    if (ldl < std::max(1, K) || ldl % 4) return mp_arg_fail(6, "ldl must be >= K and a multiple of 4");
    if (K > 0 && N > 0 && !dU) return mp_arg_fail(7, "U is NULL");
    if (ldu < std::max(1, N) || ldu % 4) return mp_arg_fail(8, "ldu must be >= N and a multiple of 4");
    if (M > 0 && N > 0 && !dC) return mp_arg_fail(9, "C is NULL");
    if (ldc < std::max(1, N) || ldc % 4) return mp_arg_fail(10, "ldc must be >= N and a multiple of 4");
    const size_t need = mp_lowp_gemm_workspace_bytes(M, N, K, prec);
    if (!work) return mp_arg_fail(11, "workspace is NULL");
    if (work_bytes < need) return mp_arg_fail(12, "workspace too small");
    if (M == 0 || N == 0 || K == 0) return 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    size_t off = 0;
    StatusBlock *sb = at<StatusBlock>(work, carve(off, sizeof(StatusBlock)));
    void *tcws = at<void>(work, carve(off, tc_workspace_bytes(std::max(M, N), K, prec)));
    MP_CUDA_TRY(cudaMemsetAsync(sb, 0, sizeof(StatusBlock), s));
    if (prec == MP_PREC_FP32) {
        MP_CUDA_TRY(launch_gemm_sub<float>(M, N, K, dL, ldl, dU, ldu, dC, ldc, s));
    } else {
        MP_CUDA_TRY(tc_trailing_update(prec, M, N, K, dL, ldl, dU, ldu, dC, ldc, tcws, &sb->st, s));
    }
    StatusBlock h;
    MP_CUDA_TRY(cudaMemcpyAsync(&h, sb, sizeof h, cudaMemcpyDeviceToHost, s));
    MP_CUDA_TRY(cudaStreamSynchronize(s));
    if (h.st.flags & MP_FLAG_TIMEOUT) {
        mp_set_error("tensor-core update: a bounded wait gave up");
        return -1000 - (int)cudaErrorLaunchTimeout;
    }
    return 0;
}

// ---------------------------------------------------------------------------
// self-test of the bounded waits' timeout path
// ---------------------------------------------------------------------------
extern "C" size_t mp_selftest_workspace_bytes(void) { return 256; }

extern "C" int mp_selftest_wait_timeout(int site, unsigned long long limit_ns, void *work, size_t work_bytes,
                                        unsigned *flags, int *site_out, int *passed, void *stream) {
    g_err[0] = 0;
    if (site < 2 || site > 4) return mp_arg_fail(1, "site must be 2 (grid barrier), 3 or 4 (mbarrier waits)");
    if (limit_ns < 1 || limit_ns > 1000000000ULL) return mp_arg_fail(2, "limit_ns must be in [1, 1e9]");
    if (!work) return mp_arg_fail(3, "workspace is NULL");
    if (work_bytes < mp_selftest_workspace_bytes()) return mp_arg_fail(4, "workspace too small");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char *w = static_cast<char *>(work);
    MpDevStatus *st = reinterpret_cast<MpDevStatus *>(w);
    unsigned *bar = reinterpret_cast<unsigned *>(w + 64);
    int *dpassed = reinterpret_cast<int *>(w + 128);
    int *abort_flag = reinterpret_cast<int *>(w + 192);
    MP_CUDA_TRY(cudaMemsetAsync(work, 0, mp_selftest_workspace_bytes(), s));
    if (site == 2) MP_CUDA_TRY(launch_selftest_grid_barrier(bar, st, limit_ns, dpassed, s));
    else if (site == 3) MP_CUDA_TRY(launch_selftest_panel_mbar(st, limit_ns, s));
    else MP_CUDA_TRY(launch_selftest_tc_mbar(st, abort_flag, limit_ns, s));
    MpDevStatus h;
    int hp = 0;
    MP_CUDA_TRY(cudaMemcpyAsync(&h, st, sizeof h, cudaMemcpyDeviceToHost, s));
    MP_CUDA_TRY(cudaMemcpyAsync(&hp, dpassed, sizeof hp, cudaMemcpyDeviceToHost, s));
    MP_CUDA_TRY(cudaStreamSynchronize(s));
    if (flags) *flags = h.flags;
    if (site_out) *site_out = h.timeout_site;
    if (passed) *passed = hp;
    return 0;
}

// ---------------------------------------------------------------------------
// extra-precise refinement (Section 5: QDGESV)
// ---------------------------------------------------------------------------
namespace {
mp_opts dd_opts() {
    mp_opts o;
    mp_default_opts(&o);
    o.prec = MP_PREC_FP64;
    return o;
}
size_t dd_part_bytes(int n, int nrhs) {
    return (size_t)residual_dd_ksplit(std::max(n, 1)) * (size_t)std::max(n, 1) * (size_t)std::max(nrhs, 1) *
           sizeof(double);
}
}  // namespace

extern "C" size_t mp_gesv_dd_workspace_bytes(int n, int nrhs) {
    if (n < 0 || nrhs < 0) return 0;
    const mp_opts o = dd_opts();
    return make_layout(n, nrhs, o, true).total + 2 * align_up(dd_part_bytes(n, nrhs), 256);
}

extern "C" int mp_gesv_dd(int n, int nrhs, const double *dA, int lda, const double *dB, int ldb, double *dXhi,
                          double *dXlo, int ldx, int32_t *dipiv, int itermax, void *work, size_t work_bytes,
                          mp_stats *stats, void *stream) {
    g_err[0] = 0;
    if (n < 0) return mp_arg_fail(1, "n < 0");
    if (nrhs < 0 || nrhs > kMaxRhs) return mp_arg_fail(2, "nrhs must be in [0, 8]");
    if (n > 65536) return mp_arg_fail(1, "n > 65536 is not supported");
    if (n > 0 && !dA) return mp_arg_fail(3, "A is NULL");
    if (lda < std::max(1, n)) return mp_arg_fail(4, "lda < max(1, n)");
    if (n > 0 && nrhs > 0 && !dB) return mp_arg_fail(5, "B is NULL");
    if (ldb < std::max(1, n)) return mp_arg_fail(6, "ldb < max(1, n)");
    if (n > 0 && nrhs > 0 && !dXhi) return mp_arg_fail(7, "Xhi is NULL");
    if (n > 0 && nrhs > 0 && !dXlo) return mp_arg_fail(8, "Xlo is NULL");
    if (ldx < std::max(1, n)) return mp_arg_fail(9, "ldx < max(1, n)");
    if (n > 0 && !dipiv) return mp_arg_fail(10, "ipiv is NULL");
    if (itermax < 0) return mp_arg_fail(11, "itermax < 0");
    if (stats) std::memset(stats, 0, sizeof(*stats));
    if (n == 0 || nrhs == 0) return 0;
    const mp_opts o = dd_opts();
    Layout L = make_layout(n, nrhs, o, true);
    if (!work) return mp_arg_fail(12, "workspace is NULL");
    if (work_bytes < mp_gesv_dd_workspace_bytes(n, nrhs)) return mp_arg_fail(13, "workspace too small");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double *part_hi = at<double>(work, L.total);
    double *part_lo = at<double>(work, L.total + align_up(dd_part_bytes(n, nrhs), 256));
    const int ks = residual_dd_ksplit(n);
    Solve S{n, nrhs, dA, lda, dB, ldb, dXhi, ldx, work, L, s, at<StatusBlock>(work, L.status), 0, false};
    const bool timing = stats != nullptr;
    cudaEvent_t ev[4] = {};
    if (timing)
        for (auto &e : ev) MP_CUDA_TRY(cudaEventCreate(&e));
    auto mark = [&](int i) { if (timing) cudaEventRecord(ev[i], s); };
    mark(0);
    MP_CUDA_TRY(cudaMemsetAsync(S.sb, 0, sizeof(StatusBlock), s));
    MP_CUDA_TRY(cudaMemsetAsync(at<double>(work, L.rowsum), 0, sizeof(double) * n, s));
    if (reset_sync(S)) return -1000;
    MP_CUDA_TRY(launch_convert_transpose<double>(n, dA, lda, at<double>(work, L.W), L.ldw, at<double>(work, L.rowsum),
                                                 &S.sb->st, s));
    MP_CUDA_TRY(launch_max_reduce(n, at<double>(work, L.rowsum), &S.sb->st.anorm, s));
    MP_CUDA_TRY(launch_col_absmax(n, nrhs, dB, ldb, S.sb->bnorm, &S.sb->st, s));
    mark(1);
    int info = 0, e;
    uint32_t fflags = 0, flags = 0;
    if ((e = factor<double>(S, MP_PREC_FP32, std::min(L.nb, 256), &info, &fflags))) return e;
    mark(2);
    flags |= fflags & MP_FLAG_NONFINITE_INPUT;
    MP_CUDA_TRY(cudaMemcpyAsync(dipiv, at<int32_t>(work, L.ipiv), sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
    int it = 0;
    if (info == 0 && !(flags & MP_FLAG_NONFINITE_INPUT)) {
        // x_0 = (LU)^{-1} P b in FP64, x_lo = 0
        MP_CUDA_TRY(cudaMemsetAsync(S.sb->znorm, 0, sizeof(double) * kMaxRhs, s));
        if ((e = lowp_solve<double>(S, dB, ldb, S.sb->bnorm, nrhs))) return e;
        MP_CUDA_TRY(launch_update_dd(n, nrhs, at<double>(work, L.Z), n, S.sb->bnorm, dXhi, dXlo, ldx, S.sb->znorm, 1, s));
        double zprev[kMaxRhs] = {0};
        const double floor = std::ldexp(1.0, -100);
        for (;;) {
            // r = b - A (x_hi + x_lo) accumulated in double-double, rounded to FP64
            MP_CUDA_TRY(cudaMemsetAsync(S.sb->rnorm, 0, sizeof(double) * 2 * kMaxRhs, s));
            {
                MpProfScope ps(MP_KC_RESIDUAL, 8.0 * n * n + 24.0 * n * nrhs, s);
                MP_CUDA_TRY(launch_residual_dd(n, nrhs, dA, lda, dXhi, dXlo, ldx, dB, ldb, part_hi, part_lo, ks,
                                               at<double>(work, L.R), n, S.sb->rnorm, S.sb->xnorm, s));
            }
            StatusBlock h;
            if ((e = read_status(S, h))) return e;
            // a column is done when its last correction reached the
            // double-double floor or stopped shrinking (the accuracy the
            // residual allows); the loop also ends at itermax corrections
            bool done = true, nonfinite = false;
            double worst = 0.0;
            for (int c = 0; c < nrhs; ++c) {
                const double den = h.st.anorm * h.xnorm[c] + h.bnorm[c];
                const double b = den > 0.0 ? h.rnorm[c] / den : (h.rnorm[c] > 0.0 ? INFINITY : 0.0);
                worst = std::max(worst, std::isnan(b) ? INFINITY : b);
                if (!std::isfinite(h.rnorm[c]) || !std::isfinite(h.xnorm[c])) nonfinite = true;
                const bool c_done = h.rnorm[c] == 0.0 || h.znorm[c] <= floor * h.xnorm[c] ||
                                    (it >= 2 && h.znorm[c] > 0.5 * zprev[c]);
                if (!c_done) done = false;
            }
            if (stats) {
                if (stats->nhist < 32) stats->hist[stats->nhist++] = worst;
                stats->bwd_err = worst;
            }
            if (nonfinite) { flags |= MP_FLAG_LOWP_BREAKDOWN; break; }
            if (done) break;
            if (it >= itermax) { flags |= MP_FLAG_NOT_CONVERGED; break; }
            std::memcpy(zprev, h.znorm, sizeof zprev);
            if ((e = lowp_solve<double>(S, at<double>(work, L.R), n, S.sb->rnorm, nrhs))) return e;
            MP_CUDA_TRY(cudaMemsetAsync(S.sb->znorm, 0, sizeof(double) * kMaxRhs, s));
            MP_CUDA_TRY(launch_update_dd(n, nrhs, at<double>(work, L.Z), n, S.sb->rnorm, dXhi, dXlo, ldx, S.sb->znorm,
                                         0, s));
            ++it;
        }
    }
    mark(3);
    MP_CUDA_TRY(cudaStreamSynchronize(s));
    if (stats) {
        stats->iter = it;
        stats->flags = flags;
        stats->info = info;
        cudaEventElapsedTime(&stats->ms_convert, ev[0], ev[1]);
        cudaEventElapsedTime(&stats->ms_factor, ev[1], ev[2]);
        cudaEventElapsedTime(&stats->ms_refine, ev[2], ev[3]);
    }
    if (timing)
        for (auto &x : ev) cudaEventDestroy(x);
    return info;
}
