// sparse.cu -- the mixed-precision inner-outer iterative method of
// Section 2.2 (Algorithm 2): FGMRES(m_out) in FP64 whose preconditioner is
// one cycle of GMRES(m_in) in single precision (GMRES_SP), on a sparse matrix
// in CSR form.  The paper's point is that the inner solver works on a cheaper
// approximation of the operator: here the FP32 copy of the matrix values and
// FP32 vectors, half the bytes per stored entry and per basis vector.
//
// GB300 design.  One restart cycle of the outer method -- the residual and
// accuracy test, up to m_out outer steps, each with a whole inner GMRES cycle,
// the outer least-squares solve and the update of x -- is ONE cooperative
// launch.  Every CTA owns a contiguous block of rows, and the grid meets at
// bounded grid barriers where a step needs data from other rows (the sparse
// product) or a global sum (dot products, norms).  The matrix (26 MB at the
// largest stand-in) and the basis vectors stay in the 129 MB L2 across steps,
// so a cycle is bound by barrier latency and L2 bandwidth, not by launches.
//
//   sparse product    L lanes per row (L = 4, 8 or 16 from the mean row
//                     length); values and vector in the working precision
//   orthogonalisation classical Gram-Schmidt applied twice (CGS2): all dot
//                     products of a pass in one reduction (the paper's
//                     modified Gram-Schmidt needs k dependent reductions);
//                     the norm after the second pass comes with it as
//                     ||w||^2 - sum h2_i^2 (h2 is at rounding level after the
//                     first pass, so nothing cancels)
//   reductions        a warp per basis vector inside a CTA; the CTA partials
//                     go to a buffer that alternates between phases and are
//                     summed after the barrier by every CTA in one fixed
//                     order, so every CTA holds identical values (data written
//                     by other CTAs is read past L1)
//   small problem     Givens rotations and back substitution by thread 0 of
//                     CTA 0, which publishes the stop decision and y before
//                     the next barrier
// The next step's sparse product reads the unnormalised vector w (complete
// at the barrier after its last update) and scales its rows by 1 / ||w||, so
// an inner step needs three grid barriers.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "common.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxM = 320;      // largest m_in / m_out (Table 3 goes up to 300)
constexpr int kMaxGrid = 1024;  // largest cooperative grid (sizes the partial sums)
constexpr int kStageBytes = 160 * 1024;  // staged x: 40960 FP32 or 20480 FP64 columns per CTA
constexpr int kRsmBytes = 16 * 1024;     // an R in shared memory: m <= 44 (FP64) or 63 (FP32)

enum Mode { kCycle = 0, kInnerOnly = 1 };

// Control block: written by CTA 0 (stop decisions, results) or by atomics,
// read by every CTA after the next grid barrier and by the host after a launch.
struct SpCtrl {
    int stop;          // the current (inner or outer) cycle ends after this step
    int steps;         // steps of the current cycle so far
    int converged;     // the accuracy test passed at the start of this launch
    int outer_steps;   // outer steps of this launch
    int inner_steps;   // inner steps of this launch
    int pad[3];
    double bwd;        // backward error of x at the start of this launch
    double est;        // last residual estimate (outer, or inner in kInnerOnly)
    double rmax, xmax; // max |r|, max |x| (atomic maxima; zeroed before a launch)
    double anorm, bnorm;
};

struct SpArgs {
    int n, mode, m_in, m_out, inner;  // inner: 0 FP32, 1 FP64, 2 none (plain restarted GMRES)
    long ld;              // stride of the basis vectors (n rounded up to 32)
    int stage_bytes;      // dynamic shared memory for the staged x
    const int *indptr, *indices;
    const double *val64;
    const void *valin;    // values in the inner precision (val64 itself for FP64)
    const double *b;
    double *x;
    double tol, stop_rel_in;
    void *Vin;            // m_in vectors of n, inner precision (normalised basis)
    void *Win;            // 2 vectors of n, inner precision (unnormalised w by step parity)
    double *Vout;         // m_out + 1 vectors of n
    double *Zout;         // m_out vectors of n
    double *W64;          // 2 vectors of n: the residual, the outer w
    unsigned char *part;  // 2 buffers of kMaxGrid x pstride 8-byte slots
    int pstride;
    double *Rout, *gout, *csout, *snout, *yout;  // outer small problem (CTA 0)
    void *Rin, *gin, *csin, *snin, *yin;         // inner small problem, inner precision
    SpCtrl *ctrl;
    unsigned *bar;        // grid barrier: count, generation
    MpDevStatus *st;
    const double *rhs_inner;  // kInnerOnly: right-hand side (FP64)
    double *z_inner;          // kInnerOnly: result (FP64)
};

template <typename T>
__device__ __forceinline__ T *part_buf(const SpArgs &a, int phase) {
    return reinterpret_cast<T *>(a.part + (size_t)(phase & 1) * kMaxGrid * a.pstride * 8);
}

// Sum over the grid of the CTA partials part[cta][0..k), in a fixed order:
// an octet (8 lanes) per entry, lane l adding CTAs l, l + 8, ..., the octet's
// sums combined by a fixed shuffle tree.  out (shared) gets the k sums in
// every CTA.
template <typename T>
__device__ void grid_sum(const T *part, int pstride, int k, T *out) {
    const int tid = threadIdx.x, oct = tid >> 3, l = tid & 7;
    const int G = gridDim.x;
    for (int i0 = 0; i0 < k; i0 += kThreads / 8) {
        const int i = i0 + oct;
        T s = T(0);
        if (i < k)
            for (int c = l; c < G; c += 8) s += __ldcg(part + (long)c * pstride + i);
        s += __shfl_xor_sync(0xffffffffu, s, 1);
        s += __shfl_xor_sync(0xffffffffu, s, 2);
        s += __shfl_xor_sync(0xffffffffu, s, 4);
        if (i < k && l == 0) out[i] = s;
    }
    __syncthreads();
}

// 16-byte vectors of the working precision.  Basis vectors are stored with a
// stride that is a multiple of 32 elements and every CTA's row block starts
// at a multiple of 32, so a CTA's rows are 16-byte vectors except for a
// ragged tail at n (last CTA only).
template <typename T> struct Vec;
template <> struct Vec<float> {
    using type = float4;
    __device__ __forceinline__ static float dot(float4 a, float4 b, float s) {
        return fmaf(a.w, b.w, fmaf(a.z, b.z, fmaf(a.y, b.y, fmaf(a.x, b.x, s))));
    }
    __device__ __forceinline__ static float4 axpy(float h, float4 v, float4 w) {
        return make_float4(fmaf(h, v.x, w.x), fmaf(h, v.y, w.y), fmaf(h, v.z, w.z), fmaf(h, v.w, w.w));
    }
};
template <> struct Vec<double> {
    using type = double2;
    __device__ __forceinline__ static double dot(double2 a, double2 b, double s) {
        return fma(a.y, b.y, fma(a.x, b.x, s));
    }
    __device__ __forceinline__ static double2 axpy(double h, double2 v, double2 w) {
        return make_double2(fma(h, v.x, w.x), fma(h, v.y, w.y));
    }
};

// part_cta[i] = sum over this CTA's rows of w[row] v_i[row], i < k (a warp
// per vector, lanes over 16-byte pieces with two in flight, shuffle tree);
// with norm, part_cta[k] = the sum of w[row]^2.
template <typename T>
__device__ void cta_dots(const T *w, const T *V, long ldv, int k, int r0, int r1, T *part_cta, bool norm) {
    using VT = typename Vec<T>::type;
    constexpr int VW = 16 / sizeof(T);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kk = k + (norm ? 1 : 0);
    const int nv = (r1 - r0) / VW, tail0 = r0 + nv * VW;
    const VT *w4 = reinterpret_cast<const VT *>(w + r0);
    for (int i = warp; i < kk; i += kWarps) {
        const T *v = i < k ? V + (long)i * ldv : w;
        const VT *v4 = reinterpret_cast<const VT *>(v + r0);
        T s0 = T(0), s1 = T(0);
        int q = lane;
        for (; q + 32 < nv; q += 64) {
            const VT a0 = w4[q], b0 = v4[q], a1 = w4[q + 32], b1 = v4[q + 32];
            s0 = Vec<T>::dot(a0, b0, s0);
            s1 = Vec<T>::dot(a1, b1, s1);
        }
        if (q < nv) s0 = Vec<T>::dot(w4[q], v4[q], s0);
        for (int row = tail0 + lane; row < r1; row += 32) s0 = fma(w[row], v[row], s0);
        T s = s0 + s1;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (lane == 0) part_cta[i] = s;
    }
}

// w -= sum_{i<k} h_i v_i on this CTA's rows (h in shared memory), a 16-byte
// piece per thread.
template <typename T>
__device__ void cta_update(T *w, const T *V, long ldv, int k, const T *h, int r0, int r1) {
    using VT = typename Vec<T>::type;
    constexpr int VW = 16 / sizeof(T);
    const int nv = (r1 - r0) / VW, tail0 = r0 + nv * VW;
    VT *w4 = reinterpret_cast<VT *>(w + r0);
    for (int q = threadIdx.x; q < nv; q += kThreads) {
        VT acc = w4[q];
        for (int i = 0; i < k; ++i) acc = Vec<T>::axpy(-h[i], reinterpret_cast<const VT *>(V + (long)i * ldv + r0)[q], acc);
        w4[q] = acc;
    }
    for (int row = tail0 + threadIdx.x; row < r1; row += kThreads) {
        T acc = w[row];
        for (int i = 0; i < k; ++i) acc = fma(-h[i], V[(long)i * ldv + row], acc);
        w[row] = acc;
    }
}

// Columns [c0, c1) of x into shared memory xs (xs[c - c0a], c0a = c0 rounded
// down to a 16-byte piece), coalesced, past L1 (other CTAs wrote x in this
// launch): 16-byte pieces while they lie below c1, elements after.
template <typename T>
__device__ void stage_x(const T *x, int c0, int c1, T *xs) {
    using VT = typename Vec<T>::type;
    constexpr int VW = 16 / sizeof(T);
    const int c0a = c0 / VW * VW;
    const int vb = c1 / VW * VW > c0a ? c1 / VW * VW : c0a;
    const bool vec = (reinterpret_cast<uintptr_t>(x) & 15) == 0;
    if (vec) {
        for (int q = threadIdx.x; q < (vb - c0a) / VW; q += kThreads)
            reinterpret_cast<VT *>(xs)[q] = __ldcg(reinterpret_cast<const VT *>(x + c0a) + q);
        for (int c = vb + threadIdx.x; c < c1; c += kThreads) xs[c - c0a] = __ldcg(x + c);
    } else {
        for (int c = c0a + threadIdx.x; c < c1; c += kThreads) xs[c - c0a] = __ldcg(x + c);
    }
    __syncthreads();
}

// Products of one row's entries e0 + sub, e0 + sub + L, ... below e1 with x
// (staged in xs when set, else from global memory past L1), two in flight.
template <typename T, typename TV, int L>
__device__ __forceinline__ T row_dot(const int *__restrict__ indices, const TV *__restrict__ val, const T *x,
                                     const T *xs, int xoff, int e0, int e1) {
    T s0 = T(0), s1 = T(0);
    int e = e0;
    if (xs) {
        for (; e + L < e1; e += 2 * L) {
            s0 = fma((T)val[e], xs[indices[e] - xoff], s0);
            s1 = fma((T)val[e + L], xs[indices[e + L] - xoff], s1);
        }
        if (e < e1) s0 = fma((T)val[e], xs[indices[e] - xoff], s0);
    } else {
        for (; e + L < e1; e += 2 * L) {
            s0 = fma((T)val[e], __ldcg(x + indices[e]), s0);
            s1 = fma((T)val[e + L], __ldcg(x + indices[e + L]), s1);
        }
        if (e < e1) s0 = fma((T)val[e], __ldcg(x + indices[e]), s0);
    }
    return s0 + s1;
}

// y[row] = scale * sum_l a_l x[col_l] for the rows [r0, r1), L lanes per row,
// in precision T (values converted from TV, i.e. rounded when TV is wider);
// with b, y[row] = b[row] - sum (the residual).  A lane group takes two rows
// per pass (their loads in flight together) and fetches the next pass's row
// pointers while it works.
template <typename T, typename TV, int L>
__device__ void spmv_rows(const int *__restrict__ indptr, const int *__restrict__ indices, const TV *__restrict__ val,
                          const T *x, const T *xs, int xoff, T *y, int r0, int r1, T scale,
                          const double *__restrict__ b) {
    const int sub = threadIdx.x % L, grp = threadIdx.x / L;
    constexpr int GROUPS = kThreads / L;
    int ra = r0 + grp, rb = ra + GROUPS;
    int pa0 = ra < r1 ? indptr[ra] : 0, pa1 = ra < r1 ? indptr[ra + 1] : 0;
    int pb0 = rb < r1 ? indptr[rb] : 0, pb1 = rb < r1 ? indptr[rb + 1] : 0;
    for (int row0 = r0; row0 < r1; row0 += 2 * GROUPS) {
        // the next pass's row pointers
        const int na = ra + 2 * GROUPS, nb = rb + 2 * GROUPS;
        const int qa0 = na < r1 ? indptr[na] : 0, qa1 = na < r1 ? indptr[na + 1] : 0;
        const int qb0 = nb < r1 ? indptr[nb] : 0, qb1 = nb < r1 ? indptr[nb + 1] : 0;
        T sa = row_dot<T, TV, L>(indices, val, x, xs, xoff, pa0 + sub, pa1);
        T sb = row_dot<T, TV, L>(indices, val, x, xs, xoff, pb0 + sub, pb1);
#pragma unroll
        for (int off = L / 2; off > 0; off >>= 1) {
            sa += __shfl_xor_sync(0xffffffffu, sa, off);
            sb += __shfl_xor_sync(0xffffffffu, sb, off);
        }
        if (sub == 0) {
            if (ra < r1) y[ra] = b ? (T)(b[ra] - (double)sa) : sa * scale;
            if (rb < r1) y[rb] = b ? (T)(b[rb] - (double)sb) : sb * scale;
        }
        ra = na;
        rb = nb;
        pa0 = qa0;
        pa1 = qa1;
        pb0 = qb0;
        pb1 = qb1;
    }
}

// The columns this CTA's rows reference, and whether x restricted to them
// fits the staging area: the sparse products then gather from shared memory.
struct ColSpan {
    int c0, c1, xoff;
    bool fits32, fits64;
};
__device__ ColSpan col_span(const int *indptr, const int *indices, int r0, int r1, int stage_bytes, int *red) {
    int lo = INT_MAX, hi = -1;
    if (r1 > r0)
        for (int e = indptr[r0] + threadIdx.x; e < indptr[r1]; e += kThreads) {
            const int c = indices[e];
            lo = min(lo, c);
            hi = max(hi, c);
        }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, off));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, off));
    }
    if ((threadIdx.x & 31) == 0) {
        red[threadIdx.x >> 5] = lo;
        red[kWarps + (threadIdx.x >> 5)] = hi;
    }
    __syncthreads();
    ColSpan cs;
    lo = INT_MAX;
    hi = -1;
    for (int w = 0; w < kWarps; ++w) {
        lo = min(lo, red[w]);
        hi = max(hi, red[kWarps + w]);
    }
    __syncthreads();
    if (hi < lo) lo = hi = 0;  // no entries
    cs.c0 = lo;
    cs.c1 = hi + 1;
    cs.xoff = lo / 4 * 4;  // the FP32 staging's rounding (FP64 rounds to 2: recomputed there)
    const long span = (long)cs.c1 - lo / 4 * 4 + 4;
    cs.fits32 = span * 4 <= stage_bytes;
    cs.fits64 = span * 8 <= stage_bytes;
    return cs;
}

// Givens rotation (c, s) with c a + s b = hypot(a, b) and -s a + c b = 0.
template <typename T>
__device__ __forceinline__ void rotation(T a, T b, T &c, T &s) {
    const T r = hypot(a, b);
    if (r == T(0)) {
        c = T(1);
        s = T(0);
    } else {
        c = a / r;
        s = b / r;
    }
}

// Thread 0 of CTA 0: column j of the Hessenberg matrix (h1 + h2 above the
// diagonal, hnext below it) into the rotated R (column-major, ld ldr), the
// earlier rotations, the new one, g; returns the residual estimate |g[j+1]|.
template <typename T>
__device__ T givens_step(T *R, T *g, T *cs, T *sn, const T *h1, const T *h2, T hnext, int j, int ldr) {
    T *col = R + (long)j * ldr;
    for (int i = 0; i <= j; ++i) col[i] = h1[i] + h2[i];
    col[j + 1] = hnext;
    for (int i = 0; i < j; ++i) {
        const T p = col[i], q = col[i + 1];
        col[i] = cs[i] * p + sn[i] * q;
        col[i + 1] = -sn[i] * p + cs[i] * q;
    }
    rotation(col[j], col[j + 1], cs[j], sn[j]);
    col[j] = cs[j] * col[j] + sn[j] * col[j + 1];
    col[j + 1] = T(0);
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    return fabs(g[j + 1]);
}

// Back substitution R y = g over the first `steps` columns (thread 0, CTA 0).
template <typename T>
__device__ void back_solve(const T *R, const T *g, T *y, int steps, int ldr) {
    for (int i = steps - 1; i >= 0; --i) {
        T acc = g[i];
        for (int l = i + 1; l < steps; ++l) acc -= R[(long)l * ldr + i] * y[l];
        y[i] = acc / R[(long)i * ldr + i];
    }
}

// The Arnoldi steps shared by the inner and the outer loop: CGS2 of wn
// against the basis V (k vectors, own rows), the two reductions, the final
// update of wn (own rows) and hnext.  h1, h2 (shared) get the coefficients.
// Returns false if a grid barrier timed out.
template <typename T>
__device__ bool cgs2(const SpArgs &a, T *wn, const T *V, int k, int r0, int r1, int &phase, bool &abort_s, T *h1,
                     T *h2, T &hnext) {
    const long ld = a.ld;
    const int ps = a.pstride;
    cta_dots<T>(wn, V, ld, k, r0, r1, part_buf<T>(a, phase) + (long)blockIdx.x * ps, false);
    if (!grid_barrier(a.bar, a.bar + 1, a.st, &abort_s)) return false;
    grid_sum<T>(part_buf<T>(a, phase), ps, k, h1);
    ++phase;
    cta_update<T>(wn, V, ld, k, h1, r0, r1);
    __syncthreads();
    cta_dots<T>(wn, V, ld, k, r0, r1, part_buf<T>(a, phase) + (long)blockIdx.x * ps, true);
    if (!grid_barrier(a.bar, a.bar + 1, a.st, &abort_s)) return false;
    grid_sum<T>(part_buf<T>(a, phase), ps, k + 1, h2);
    ++phase;
    cta_update<T>(wn, V, ld, k, h2, r0, r1);
    T nrm2 = h2[k];
    for (int i = 0; i < k; ++i) nrm2 -= h2[i] * h2[i];
    hnext = sqrt(nrm2 > T(0) ? nrm2 : T(0));
    return true;
}

// One cycle of GMRES(m_in) in precision T for A z = v from z = 0 (the inner
// solver of Algorithm 2); z written to zdst (FP64) on this CTA's rows.
// Returns false if a grid barrier timed out.
template <typename T, int L>
__device__ bool inner_cycle(const SpArgs &a, const double *v, double *zdst, int r0, int r1, int &phase,
                            bool &abort_s, T *h1, T *h2, int *steps_out, T *beta_out, const ColSpan &span,
                            T *xstage, T *R, T *g, T *cs, T *sn) {
    const bool stage_in = sizeof(T) == 4 ? span.fits32 : span.fits64;
    const int m = a.m_in, tid = threadIdx.x, ps = a.pstride;
    const long ld = a.ld;
    const bool lead = blockIdx.x == 0 && tid == 0;
    T *Vin = reinterpret_cast<T *>(a.Vin);
    T *Win = reinterpret_cast<T *>(a.Win);
    const T *val = reinterpret_cast<const T *>(a.valin);
    T *y = reinterpret_cast<T *>(a.yin);
    // r0 = fl_T(v), unnormalised, into Win[0], and its norm
    for (int row = r0 + tid; row < r1; row += kThreads) Win[row] = (T)v[row];
    __syncthreads();
    cta_dots<T>(Win, Win, ld, 0, r0, r1, part_buf<T>(a, phase) + (long)blockIdx.x * ps, true);
    if (!grid_barrier(a.bar, a.bar + 1, a.st, &abort_s)) return false;
    grid_sum<T>(part_buf<T>(a, phase), ps, 1, h1);
    ++phase;
    const T beta = sqrt(h1[0]);
    *beta_out = beta;
    int steps = 0;
    if (beta > T(0)) {
        if (lead) g[0] = beta;
        T hprev = beta;
        const T stop_abs = (T)a.stop_rel_in * beta;
        for (int j = 0; j < m; ++j) {
            const T *wp = Win + (j & 1) * ld;  // w_j unnormalised, complete on every row
            T *wn = Win + ((j + 1) & 1) * ld;
            T *vj = Vin + j * ld;
            const T inv = T(1) / hprev;
            for (int row = r0 + tid; row < r1; row += kThreads) vj[row] = wp[row] * inv;
            const T *xs = nullptr;
            int xoff = 0;
            if (stage_in) {
                stage_x<T>(wp, span.c0, span.c1, xstage);
                xs = xstage;
                xoff = span.c0 / (16 / (int)sizeof(T)) * (16 / (int)sizeof(T));
            }
            spmv_rows<T, T, L>(a.indptr, a.indices, val, wp, xs, xoff, wn, r0, r1, inv, nullptr);
            __syncthreads();
            T hnext;
            if (!cgs2<T>(a, wn, Vin, j + 1, r0, r1, phase, abort_s, h1, h2, hnext)) return false;
            if (lead) {
                const T est = givens_step<T>(R, g, cs, sn, h1, h2, hnext, j, m + 1);
                const bool stop = hnext == T(0) || est <= stop_abs || j + 1 == m;
                if (stop) back_solve<T>(R, g, y, j + 1, m + 1);
                a.ctrl->stop = stop ? 1 : 0;
                a.ctrl->est = (double)est;
            }
            // w complete on every row; the decision (and y) published
            if (!grid_barrier(a.bar, a.bar + 1, a.st, &abort_s)) return false;
            steps = j + 1;
            if (*(volatile int *)&a.ctrl->stop) break;
            hprev = hnext;
        }
        // z = V y on this CTA's rows (working precision), widened to FP64
        for (int i = tid; i < steps; i += kThreads) h1[i] = __ldcg(y + i);
        __syncthreads();
        for (int row = r0 + tid; row < r1; row += kThreads) {
            T z = T(0);
            for (int i = 0; i < steps; ++i) z = fma(h1[i], Vin[i * ld + row], z);
            zdst[row] = (double)z;
        }
    } else {
        for (int row = r0 + tid; row < r1; row += kThreads) zdst[row] = 0.0;
    }
    *steps_out = steps;
    __syncthreads();  // h1 is reused by the caller
    return true;
}

// One restart cycle of FGMRES(m_out)-GMRES(m_in) (mode kCycle), or one inner
// cycle alone (mode kInnerOnly, for the parity tests).  Cooperative launch.
template <typename Tin, int L>
__global__ void __launch_bounds__(kThreads) fgmres_kernel(const SpArgs a) {
    __shared__ double hd1[kMaxM + 2], hd2[kMaxM + 2];
    __shared__ Tin hi1[kMaxM + 2], hi2[kMaxM + 2];
    // the small problems' rotations and right-hand sides (CTA 0 uses them)
    __shared__ double gout_s[kMaxM + 2], csout_s[kMaxM + 2], snout_s[kMaxM + 2];
    __shared__ Tin gin_s[kMaxM + 2], csin_s[kMaxM + 2], snin_s[kMaxM + 2];
    __shared__ int red[2 * kWarps];
    __shared__ bool abort_s;
    extern __shared__ __align__(16) unsigned char dyn[];  // staged x, then the two R when they fit
    if (threadIdx.x == 0) abort_s = false;
    __syncthreads();
    const int n = a.n, tid = threadIdx.x, ps = a.pstride;
    const long ld = a.ld;
    const bool lead = blockIdx.x == 0 && tid == 0;
    // row blocks start at multiples of 32 (16-byte pieces of every vector)
    const int per = ((n + (int)gridDim.x - 1) / (int)gridDim.x + 31) / 32 * 32;
    const int r0 = min(n, (int)blockIdx.x * per), r1 = min(n, r0 + per);
    const ColSpan span = col_span(a.indptr, a.indices, r0, r1, a.stage_bytes, red);
    Tin *xs_in = reinterpret_cast<Tin *>(dyn);
    double *xs64 = reinterpret_cast<double *>(dyn);
    // R of the small problems in shared memory when it fits (else global)
    const size_t rin_bytes = sizeof(Tin) * (size_t)(a.m_in + 1) * a.m_in;
    const size_t rout_bytes = sizeof(double) * (size_t)(a.m_out + 1) * a.m_out;
    double *Rout = rout_bytes <= kRsmBytes ? reinterpret_cast<double *>(dyn + a.stage_bytes) : a.Rout;
    Tin *Rin = rin_bytes <= kRsmBytes ? reinterpret_cast<Tin *>(dyn + a.stage_bytes + kRsmBytes)
                                      : reinterpret_cast<Tin *>(a.Rin);
    int phase = 0;
    if (a.mode == kInnerOnly) {
        int steps = 0;
        Tin beta = Tin(0);
        if (!inner_cycle<Tin, L>(a, a.rhs_inner, a.z_inner, r0, r1, phase, abort_s, hi1, hi2, &steps, &beta, span,
                                 xs_in, Rin, gin_s, csin_s, snin_s))
            return;
        if (lead) a.ctrl->inner_steps = steps;
        return;
    }
    // ---- r = b - A x (FP64), the accuracy test
    double *r = a.W64, *w64 = a.W64 + ld;
    if (span.fits64) stage_x<double>(a.x, span.c0, span.c1, xs64);
    spmv_rows<double, double, L>(a.indptr, a.indices, a.val64, a.x, span.fits64 ? xs64 : nullptr, span.c0 / 2 * 2, r,
                                 r0, r1, 1.0, a.b);
    __syncthreads();
    {
        double rm = 0.0, xm = 0.0;
        for (int row = r0 + tid; row < r1; row += kThreads) {
            rm = fmax(rm, fabs(r[row]));
            xm = fmax(xm, fabs(a.x[row]));
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            rm = fmax(rm, __shfl_xor_sync(0xffffffffu, rm, off));
            xm = fmax(xm, __shfl_xor_sync(0xffffffffu, xm, off));
        }
        if ((tid & 31) == 0) {
            atomic_max_nonneg(&a.ctrl->rmax, rm);
            atomic_max_nonneg(&a.ctrl->xmax, xm);
        }
    }
    cta_dots<double>(r, r, ld, 0, r0, r1, part_buf<double>(a, phase) + (long)blockIdx.x * ps, true);
    if (!grid_barrier(a.bar, a.bar + 1, a.st, &abort_s)) return;
    grid_sum<double>(part_buf<double>(a, phase), ps, 1, hd1);
    ++phase;
    const double beta = sqrt(hd1[0]);
    const double rmax = __ldcg(&a.ctrl->rmax), xmax = __ldcg(&a.ctrl->xmax);
    const double anorm = __ldcg(&a.ctrl->anorm), bnorm = __ldcg(&a.ctrl->bnorm);
    const double den = anorm * xmax + bnorm;
    const double bwd = den > 0.0 ? rmax / den : 0.0;
    if (lead) a.ctrl->bwd = bwd;
    if (bwd <= a.tol || beta == 0.0) {
        if (lead) a.ctrl->converged = 1;
        return;
    }
    // outer steps end early once the estimate shows the accuracy test will pass
    const double xs = anorm > 0.0 ? fmax(xmax, bnorm / anorm) : xmax;
    const double tau = 0.5 * a.tol * (anorm * xs + bnorm);
    for (int row = r0 + tid; row < r1; row += kThreads) a.Vout[row] = r[row] / beta;
    if (lead) gout_s[0] = beta;
    int used = 0, inner_total = 0;
    for (int k = 0; k < a.m_out; ++k) {
        double *zk = a.Zout + k * ld;
        const double *vk = a.Vout + k * ld;
        if (a.inner == 2) {  // no preconditioner: plain restarted GMRES(m_out)
            for (int row = r0 + tid; row < r1; row += kThreads) zk[row] = vk[row];
        } else {
            int steps = 0;
            Tin bi = Tin(0);
            if (!inner_cycle<Tin, L>(a, vk, zk, r0, r1, phase, abort_s, hi1, hi2, &steps, &bi, span, xs_in, Rin,
                                     gin_s, csin_s, snin_s))
                return;
            inner_total += steps;
        }
        __syncthreads();
        if (!grid_barrier(a.bar, a.bar + 1, a.st, &abort_s)) return;  // z_k complete on every row
        if (span.fits64) stage_x<double>(zk, span.c0, span.c1, xs64);
        spmv_rows<double, double, L>(a.indptr, a.indices, a.val64, zk, span.fits64 ? xs64 : nullptr, span.c0 / 2 * 2,
                                     w64, r0, r1, 1.0, nullptr);
        __syncthreads();
        double hnext;
        if (!cgs2<double>(a, w64, a.Vout, k + 1, r0, r1, phase, abort_s, hd1, hd2, hnext)) return;
        if (lead) {
            const double est = givens_step<double>(Rout, gout_s, csout_s, snout_s, hd1, hd2, hnext, k, a.m_out + 1);
            const bool stop = hnext == 0.0 || est <= tau || k + 1 == a.m_out;
            if (stop) back_solve<double>(Rout, gout_s, a.yout, k + 1, a.m_out + 1);
            a.ctrl->stop = stop ? 1 : 0;
            a.ctrl->est = est;
        }
        if (hnext > 0.0)
            for (int row = r0 + tid; row < r1; row += kThreads) a.Vout[(k + 1) * ld + row] = w64[row] / hnext;
        if (!grid_barrier(a.bar, a.bar + 1, a.st, &abort_s)) return;  // the decision (and y) published
        used = k + 1;
        if (*(volatile int *)&a.ctrl->stop) break;
    }
    // x = x + Z y on this CTA's rows
    for (int i = tid; i < used; i += kThreads) hd1[i] = __ldcg(a.yout + i);
    __syncthreads();
    for (int row = r0 + tid; row < r1; row += kThreads) {
        double z = 0.0;
        for (int i = 0; i < used; ++i) z = fma(hd1[i], a.Zout[i * ld + row], z);
        a.x[row] = a.x[row] + z;
    }
    if (lead) {
        a.ctrl->outer_steps = used;
        a.ctrl->inner_steps = inner_total;
    }
}

// ||A||inf (row sums of |a_ij|) and ||b||inf into the control block (zeroed before).
__global__ void sparse_norms_kernel(int n, const int *__restrict__ indptr, const double *__restrict__ val,
                                    const double *__restrict__ b, SpCtrl *ctrl) {
    double am = 0.0, bm = 0.0;
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < n; row += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int e = indptr[row]; e < indptr[row + 1]; ++e) s += fabs(val[e]);
        am = fmax(am, s);
        bm = fmax(bm, fabs(b[row]));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        am = fmax(am, __shfl_xor_sync(0xffffffffu, am, off));
        bm = fmax(bm, __shfl_xor_sync(0xffffffffu, bm, off));
    }
    if ((threadIdx.x & 31) == 0) {
        atomic_max_nonneg(&ctrl->anorm, am);
        atomic_max_nonneg(&ctrl->bnorm, bm);
    }
}

// FP64 values rounded to FP32 (round to nearest even).
__global__ void values_to_f32_kernel(long nnz, const double *__restrict__ v, float *__restrict__ out) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < nnz; i += (long)gridDim.x * blockDim.x)
        out[i] = __double2float_rn(v[i]);
}

// y = A x for the step call: FP64, or FP32 with values and x rounded on the fly.
template <typename T, int L>
__global__ void __launch_bounds__(kThreads) spmv_kernel(int n, const int *indptr, const int *indices,
                                                        const double *val, const double *x, double *y) {
    const int sub = threadIdx.x % L, grp = threadIdx.x / L;
    constexpr int GROUPS = kThreads / L;
    for (int row0 = blockIdx.x * GROUPS; row0 < n; row0 += gridDim.x * GROUPS) {
        const int row = row0 + grp;
        T s = T(0);
        if (row < n)
            for (int e = indptr[row] + sub; e < indptr[row + 1]; e += L) s = fma((T)val[e], (T)x[indices[e]], s);
#pragma unroll
        for (int off = L / 2; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (row < n && sub == 0) y[row] = (double)s;
    }
}

int lanes_per_row(int n, long nnz) {
    const double avg = n > 0 ? (double)nnz / n : 0.0;
    return avg <= 12.0 ? 4 : avg <= 48.0 ? 8 : 16;
}

int sm_count() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess || sms <= 0)
        return 148;
    return sms;
}

// Workspace layout of the sparse solver.
struct SpLayout {
    size_t ctrl, bar, st, valin, Vin, Win, Vout, Zout, W64, part, Rout, gout, csout, snout, yout, Rin, gin, csin,
        snin, yin, total;
};
size_t sp_carve(size_t &off, size_t bytes) {
    off = align_up(off, 256);
    const size_t at = off;
    off += bytes;
    return at;
}
SpLayout sp_layout(int n_, long nnz, int m_in, int m_out, int inner) {
    SpLayout L{};
    const size_t n = ((size_t)n_ + 31) / 32 * 32;  // vector stride
    const size_t ein = inner == 0 ? sizeof(float) : sizeof(double);
    const size_t mi = inner == 2 ? 0 : (size_t)std::max(m_in, 1);
    size_t off = 0;
    L.ctrl = sp_carve(off, sizeof(SpCtrl));
    L.bar = sp_carve(off, 4 * sizeof(unsigned));
    L.st = sp_carve(off, sizeof(MpDevStatus));
    L.valin = sp_carve(off, inner == 0 ? sizeof(float) * (size_t)nnz : 0);
    L.Vin = sp_carve(off, ein * mi * n);
    L.Win = sp_carve(off, ein * 2 * n);
    L.Vout = sp_carve(off, sizeof(double) * (size_t)(m_out + 1) * n);
    L.Zout = sp_carve(off, sizeof(double) * (size_t)m_out * n);
    L.W64 = sp_carve(off, sizeof(double) * 2 * n);
    L.part = sp_carve(off, (size_t)2 * kMaxGrid * (kMaxM + 2) * 8);
    L.Rout = sp_carve(off, sizeof(double) * (size_t)(m_out + 1) * m_out);
    L.gout = sp_carve(off, sizeof(double) * (m_out + 1));
    L.csout = sp_carve(off, sizeof(double) * (m_out + 1));
    L.snout = sp_carve(off, sizeof(double) * (m_out + 1));
    L.yout = sp_carve(off, sizeof(double) * (m_out + 1));
    L.Rin = sp_carve(off, ein * (mi + 1) * mi);
    L.gin = sp_carve(off, ein * (mi + 1));
    L.csin = sp_carve(off, ein * (mi + 1));
    L.snin = sp_carve(off, ein * (mi + 1));
    L.yin = sp_carve(off, ein * (mi + 1));
    L.total = align_up(off, 256);
    return L;
}

template <typename Tin, int L>
cudaError_t launch_fgmres_t(const SpArgs &a, cudaStream_t s) {
    auto kern = fgmres_kernel<Tin, L>;
    const size_t smem = (size_t)kStageBytes + 2 * (size_t)kRsmBytes;
    cudaError_t e = mp_smem_attr(kern, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    // one CTA per SM: the grid barrier's cost grows with the CTA count
    int grid = std::min(sm_count(), kMaxGrid);
    grid = std::max(1, std::min(grid, (a.n + 31) / 32));
    SpArgs args = a;
    args.stage_bytes = kStageBytes;
    void *kargs[] = {(void *)&args};
    mp_note_launch();
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(kern), dim3(grid), dim3(kThreads), kargs, smem,
                                       s);
}

cudaError_t launch_fgmres(const SpArgs &a, int lanes, cudaStream_t s) {
    if (a.inner == 0) {
        if (lanes == 4) return launch_fgmres_t<float, 4>(a, s);
        if (lanes == 8) return launch_fgmres_t<float, 8>(a, s);
        return launch_fgmres_t<float, 16>(a, s);
    }
    if (lanes == 4) return launch_fgmres_t<double, 4>(a, s);
    if (lanes == 8) return launch_fgmres_t<double, 8>(a, s);
    return launch_fgmres_t<double, 16>(a, s);
}

int check_sparse_opts(const mp_sparse_opts *o, int idx) {
    if (!o) return mp_arg_fail(idx, "opts is NULL");
    if (o->m_out < 1 || o->m_out > kMaxM) return mp_arg_fail(idx, "m_out must be in [1, 320]");
    if (o->inner != MP_INNER_NONE && (o->m_in < 1 || o->m_in > kMaxM)) return mp_arg_fail(idx, "m_in must be in [1, 320]");
    if (o->inner < MP_INNER_FP32 || o->inner > MP_INNER_NONE) return mp_arg_fail(idx, "inner must be an mp_inner value");
    if (!(o->tol > 0.0) || o->max_cycles < 0) return mp_arg_fail(idx, "tol must be > 0 and max_cycles >= 0");
    return 0;
}

// Common set-up: workspace pointers, the FP32 values, the norms.
int sparse_setup(int n, long nnz, const int32_t *indptr, const int32_t *indices, const double *values,
                 const double *b, double *x, void *work, size_t work_bytes, int work_arg, const mp_sparse_opts &o,
                 SpArgs &a, SpLayout &L, cudaStream_t s) {
    L = sp_layout(n, nnz, o.m_in, o.m_out, o.inner);
    if (!work || work_bytes < L.total) return mp_arg_fail(work_arg, "workspace too small (mp_fgmres_workspace_bytes)");
    char *w = static_cast<char *>(work);
    a = SpArgs{};
    a.n = n;
    a.ld = ((long)n + 31) / 32 * 32;
    a.m_in = o.inner == MP_INNER_NONE ? 0 : o.m_in;
    a.m_out = o.m_out;
    a.inner = o.inner;
    a.indptr = indptr;
    a.indices = indices;
    a.val64 = values;
    a.valin = o.inner == MP_INNER_FP32 ? (const void *)(w + L.valin) : (const void *)values;
    a.b = b;
    a.x = x;
    a.tol = o.tol;
    // the inner cycle ends once its estimate is at its working precision's level
    a.stop_rel_in = o.inner == MP_INNER_FP32 ? 4.0 * 0x1p-24 : 4.0 * 0x1p-53;
    a.Vin = w + L.Vin;
    a.Win = w + L.Win;
    a.Vout = reinterpret_cast<double *>(w + L.Vout);
    a.Zout = reinterpret_cast<double *>(w + L.Zout);
    a.W64 = reinterpret_cast<double *>(w + L.W64);
    a.part = reinterpret_cast<unsigned char *>(w + L.part);
    a.pstride = kMaxM + 2;
    a.Rout = reinterpret_cast<double *>(w + L.Rout);
    a.gout = reinterpret_cast<double *>(w + L.gout);
    a.csout = reinterpret_cast<double *>(w + L.csout);
    a.snout = reinterpret_cast<double *>(w + L.snout);
    a.yout = reinterpret_cast<double *>(w + L.yout);
    a.Rin = w + L.Rin;
    a.gin = w + L.gin;
    a.csin = w + L.csin;
    a.snin = w + L.snin;
    a.yin = w + L.yin;
    a.ctrl = reinterpret_cast<SpCtrl *>(w + L.ctrl);
    a.bar = reinterpret_cast<unsigned *>(w + L.bar);
    a.st = reinterpret_cast<MpDevStatus *>(w + L.st);
    MP_CUDA_TRY(cudaMemsetAsync(w + L.ctrl, 0, L.valin - L.ctrl, s));  // control, barrier, status
    if (o.inner == MP_INNER_FP32 && nnz > 0) {
        mp_note_launch();
        values_to_f32_kernel<<<1024, 256, 0, s>>>(nnz, values, reinterpret_cast<float *>(w + L.valin));
        MP_CUDA_TRY(cudaGetLastError());
    }
    mp_note_launch();
    sparse_norms_kernel<<<std::max(1, std::min(1024, (n + 255) / 256)), 256, 0, s>>>(n, indptr, values, b, a.ctrl);
    MP_CUDA_TRY(cudaGetLastError());
    return 0;
}

}  // namespace

extern "C" void mp_sparse_default_opts(mp_sparse_opts *o) {
    if (!o) return;
    o->m_out = 20;
    o->m_in = 30;
    o->inner = MP_INNER_FP32;
    o->max_cycles = 100;
    o->tol = 1e-14;
}

extern "C" size_t mp_fgmres_workspace_bytes(int n, long long nnz, const mp_sparse_opts *opts) {
    mp_sparse_opts o;
    mp_sparse_default_opts(&o);
    if (opts) o = *opts;
    if (n < 0 || nnz < 0 || o.m_out < 1 || o.m_out > kMaxM || o.m_in > kMaxM) return 0;
    return sp_layout(n, (long)nnz, std::max(o.m_in, 1), o.m_out, o.inner).total;
}

extern "C" int mp_fgmres(int n, long long nnz, const int32_t *d_indptr, const int32_t *d_indices,
                         const double *d_values, const double *d_b, double *d_x, void *work, size_t work_bytes,
                         const mp_sparse_opts *opts, mp_sparse_stats *stats, void *stream) {
    if (n < 0) return mp_arg_fail(1, "n < 0");
    if (nnz < 0) return mp_arg_fail(2, "nnz < 0");
    if (n > 0 && !d_indptr) return mp_arg_fail(3, "indptr is NULL");
    if (nnz > 0 && !d_indices) return mp_arg_fail(4, "indices is NULL");
    if (nnz > 0 && !d_values) return mp_arg_fail(5, "values is NULL");
    if (n > 0 && !d_b) return mp_arg_fail(6, "b is NULL");
    if (n > 0 && !d_x) return mp_arg_fail(7, "x is NULL");
    if (int e = check_sparse_opts(opts, 10)) return e;
    const mp_sparse_opts o = *opts;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (stats) std::memset(stats, 0, sizeof(*stats));
    if (n == 0) return 0;
    SpArgs a;
    SpLayout L;
    if (int e = sparse_setup(n, (long)nnz, d_indptr, d_indices, d_values, d_b, d_x, work, work_bytes, 9, o, a, L, s))
        return e;
    MP_CUDA_TRY(cudaMemsetAsync(d_x, 0, sizeof(double) * (size_t)n, s));  // x_0 = 0
    const int lanes = lanes_per_row(n, (long)nnz);
    a.mode = kCycle;
    SpCtrl h{};
    MpDevStatus hst{};
    int cycles = 0, outer = 0, inner = 0, nh = 0;
    bool converged = false;
    for (;;) {
        // per launch: the maxima and the results start from zero
        MP_CUDA_TRY(cudaMemsetAsync(a.ctrl, 0, offsetof(SpCtrl, anorm), s));
        MP_CUDA_TRY(launch_fgmres(a, lanes, s));
        MP_CUDA_TRY(cudaMemcpyAsync(&h, a.ctrl, sizeof(SpCtrl), cudaMemcpyDeviceToHost, s));
        MP_CUDA_TRY(cudaMemcpyAsync(&hst, a.st, sizeof(MpDevStatus), cudaMemcpyDeviceToHost, s));
        MP_CUDA_TRY(cudaStreamSynchronize(s));
        if (stats && nh < 32) stats->hist[nh++] = h.bwd;
        if (hst.flags & MP_FLAG_TIMEOUT) break;
        if (h.converged) {
            converged = true;
            break;
        }
        outer += h.outer_steps;
        inner += h.inner_steps;
        if (++cycles >= o.max_cycles) break;
    }
    if (stats) {
        stats->cycles = cycles;
        stats->outer_steps = outer;
        stats->inner_steps = inner;
        stats->bwd_err = h.bwd;
        stats->nhist = nh;
        stats->flags = hst.flags | (converged ? 0u : MP_FLAG_NOT_CONVERGED);
    }
    return 0;
}

extern "C" int mp_sparse_gmres_cycle(int n, long long nnz, const int32_t *d_indptr, const int32_t *d_indices,
                                     const double *d_values, const double *d_v, double *d_z, int m, int inner,
                                     void *work, size_t work_bytes, int *steps, void *stream) {
    if (n < 0) return mp_arg_fail(1, "n < 0");
    if (nnz < 0) return mp_arg_fail(2, "nnz < 0");
    if (n > 0 && (!d_indptr || (nnz > 0 && (!d_indices || !d_values)))) return mp_arg_fail(3, "a CSR array is NULL");
    if (n > 0 && (!d_v || !d_z)) return mp_arg_fail(6, "v or z is NULL");
    if (m < 1 || m > kMaxM) return mp_arg_fail(8, "m must be in [1, 320]");
    if (inner != MP_INNER_FP32 && inner != MP_INNER_FP64) return mp_arg_fail(9, "inner must be FP32 or FP64");
    if (steps) *steps = 0;
    if (n == 0) return 0;
    mp_sparse_opts o;
    mp_sparse_default_opts(&o);
    o.m_in = m;
    o.m_out = 1;
    o.inner = inner;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    SpArgs a;
    SpLayout L;
    if (int e = sparse_setup(n, (long)nnz, d_indptr, d_indices, d_values, d_v, d_z, work, work_bytes, 11, o, a, L,
                              s))
        return e;
    a.mode = kInnerOnly;
    a.rhs_inner = d_v;
    a.z_inner = d_z;
    MP_CUDA_TRY(launch_fgmres(a, lanes_per_row(n, (long)nnz), s));
    SpCtrl h{};
    MP_CUDA_TRY(cudaMemcpyAsync(&h, a.ctrl, sizeof(SpCtrl), cudaMemcpyDeviceToHost, s));
    MP_CUDA_TRY(cudaStreamSynchronize(s));
    if (steps) *steps = h.inner_steps;
    return 0;
}

extern "C" int mp_csr_spmv(int n, long long nnz, const int32_t *d_indptr, const int32_t *d_indices,
                           const double *d_values, const double *d_x, double *d_y, int prec, void *stream) {
    if (n < 0) return mp_arg_fail(1, "n < 0");
    if (nnz < 0) return mp_arg_fail(2, "nnz < 0");
    if (n > 0 && (!d_indptr || (nnz > 0 && (!d_indices || !d_values)))) return mp_arg_fail(3, "a CSR array is NULL");
    if (n > 0 && (!d_x || !d_y)) return mp_arg_fail(6, "x or y is NULL");
    if (prec != MP_PREC_FP64 && prec != MP_PREC_FP32) return mp_arg_fail(8, "prec must be MP_PREC_FP64 or MP_PREC_FP32");
    if (n == 0) return 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int lanes = lanes_per_row(n, (long)nnz);
    const int grid = std::min(4096, (n + kThreads / lanes - 1) / (kThreads / lanes));
    mp_note_launch();
    if (prec == MP_PREC_FP64) {
        if (lanes == 4) spmv_kernel<double, 4><<<grid, kThreads, 0, s>>>(n, d_indptr, d_indices, d_values, d_x, d_y);
        else if (lanes == 8) spmv_kernel<double, 8><<<grid, kThreads, 0, s>>>(n, d_indptr, d_indices, d_values, d_x, d_y);
        else spmv_kernel<double, 16><<<grid, kThreads, 0, s>>>(n, d_indptr, d_indices, d_values, d_x, d_y);
    } else {
        if (lanes == 4) spmv_kernel<float, 4><<<grid, kThreads, 0, s>>>(n, d_indptr, d_indices, d_values, d_x, d_y);
        else if (lanes == 8) spmv_kernel<float, 8><<<grid, kThreads, 0, s>>>(n, d_indptr, d_indices, d_values, d_x, d_y);
        else spmv_kernel<float, 16><<<grid, kThreads, 0, s>>>(n, d_indptr, d_indices, d_values, d_x, d_y);
    }
    MP_CUDA_TRY(cudaGetLastError());
    return 0;
}
