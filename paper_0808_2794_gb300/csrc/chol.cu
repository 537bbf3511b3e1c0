// chol.cu -- Cholesky pieces for symmetric positive definite systems
// (Section 3.1.1: SPOTRF / SPOTRS / DSYMM take the places of SGETRF /
// SGETRS / DGEMM in Algorithm 1; Section 6 lists the Cholesky variant).
//
// The working matrix W is row-major (W[i*ldw + j] = a_ij) and only its lower
// triangle is meaningful on entry.  A = L L^T is computed in place (L in the
// lower triangle), right-looking by column blocks:
//   * leaf: the diagonal nc x nc block is factored (POTF2) and the rows
//     below it are solved against L11^T (TRSM), all in one launch;
//   * the updates between leaves and the trailing update are
//     A22 -= L21 L21^T on the lower tiles only (blas3.cu / tc_gemm.cu).
// After the factorization L^T is mirrored into the upper triangle so the
// triangular solves read both factors row-wise, as they do for LU.
#include "common.cuh"
#include "kernels.cuh"

namespace {

constexpr int kLeaf = 32;      // leaf width (columns)
constexpr int kLeafRows = 128; // rows below the diagonal block per CTA (one per thread)

// Rows [k0, n) x columns [k0, k0 + nc) of W, nc <= kLeaf.  In every CTA,
// warp 0 factors the diagonal block in registers, one row per lane, taking
// the column entries of other rows by shuffle (the same arithmetic in each
// CTA, so the copies agree bit for bit); CTA 0 writes it back.  Then each thread
// takes one row below the block and solves x L11^T = a by forward
// substitution.  A non-positive or non-finite pivot sets LOWP_BREAKDOWN and
// the first such column (1-based) in zero_pivot; the pivot is replaced by 1
// so the remaining arithmetic stays finite (the caller falls back).
template <typename T>
__global__ void __launch_bounds__(kLeafRows)
potrf_leaf_kernel(int n, int k0, int nc, T *__restrict__ W, long ldw, MpDevStatus *st) {
    __shared__ T Ls[kLeaf][kLeaf + 1];
    extern __shared__ __align__(16) unsigned char raw[];
    T(*Rs)[kLeaf + 1] = reinterpret_cast<T(*)[kLeaf + 1]>(raw);
    const int tid = threadIdx.x;
    for (int idx = tid; idx < kLeaf * kLeaf; idx += blockDim.x) {
        const int i = idx / kLeaf, j = idx % kLeaf;
        Ls[i][j] = (i < nc && j <= i) ? W[(long)(k0 + i) * ldw + k0 + j] : T(0);
    }
    // stage this CTA's rows below the block (coalesced along the row)
    const int rbase = k0 + nc + blockIdx.x * kLeafRows;
    const int nrows = max(0, min(kLeafRows, n - rbase));
    for (int idx = tid; idx < nrows * nc; idx += blockDim.x) {
        const int r = idx / nc, j = idx % nc;
        Rs[r][j] = W[(long)(rbase + r) * ldw + k0 + j];
    }
    __syncthreads();
    // POTF2 on the diagonal block, right-looking, by warp 0: lane i holds row i
    static_assert(kLeaf == 32, "one lane per row of the diagonal block");
    if (tid < 32) {
        const int i = tid;
        T b[kLeaf];
#pragma unroll
        for (int c = 0; c < kLeaf; ++c) b[c] = Ls[i][c];
#pragma unroll
        for (int j = 0; j < kLeaf; ++j) {
            if (j >= nc) break;  // uniform
            T d = __shfl_sync(0xffffffffu, b[j], j);
            if (!(d > T(0)) || !(d < T(INFINITY))) {
                if (blockIdx.x == 0 && i == 0) {
                    mp_flag(st, MP_FLAG_LOWP_BREAKDOWN);
                    atomicCAS(&st->zero_pivot, 0, k0 + j + 1);
                }
                d = T(1);
            }
            const T ljj = sqrt(d);
            if (i == j) b[j] = ljj;
            else if (i > j && i < nc) b[j] = b[j] / ljj;
            // a_ic -= l_ij l_cj for j < c <= i < nc
#pragma unroll
            for (int c = j + 1; c < kLeaf; ++c) {
                const T lcj = __shfl_sync(0xffffffffu, b[j], c);
                if (c <= i && i < nc) b[c] = fma(-b[j], lcj, b[c]);
            }
        }
#pragma unroll
        for (int c = 0; c < kLeaf; ++c) Ls[i][c] = b[c];
    }
    __syncthreads();
    if (blockIdx.x == 0)
        for (int idx = tid; idx < nc * nc; idx += blockDim.x) {
            const int i = idx / nc, j = idx % nc;
            if (j <= i) W[(long)(k0 + i) * ldw + k0 + j] = Ls[i][j];
        }
    // rows below: x_j = (a_j - sum_{p<j} x_p l_jp) / l_jj, the row in
    // registers (the loads of L are independent of the chain)
    if (tid < nrows) {
        T x[kLeaf];
#pragma unroll
        for (int j = 0; j < kLeaf; ++j) x[j] = j < nc ? Rs[tid][j] : T(0);
#pragma unroll
        for (int j = 0; j < kLeaf; ++j) {
            if (j >= nc) break;  // uniform
            T s = x[j];
#pragma unroll
            for (int p = 0; p < j; ++p) s = fma(-x[p], Ls[j][p], s);
            x[j] = s / Ls[j][j];
        }
#pragma unroll
        for (int j = 0; j < kLeaf; ++j)
            if (j < nc) Rs[tid][j] = x[j];
    }
    __syncthreads();
    for (int idx = tid; idx < nrows * nc; idx += blockDim.x) {
        const int r = idx / nc, j = idx % nc;
        W[(long)(rbase + r) * ldw + k0 + j] = Rs[r][j];
    }
}

// W[j][i] = W[i][j] for i > j (lower triangle mirrored into the upper one).
template <typename T>
__global__ void __launch_bounds__(256)
mirror_lower_kernel(int n, T *W, long ldw) {
    __shared__ T t[32][33];
    const int bi = blockIdx.y, bj = blockIdx.x;
    if (bj > bi) return;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int r = bi * 32 + ty + 8 * q, c = bj * 32 + tx;
        t[ty + 8 * q][tx] = (r < n && c < n) ? W[(long)r * ldw + c] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        // destination row bj*32 + ty + 8q, column bi*32 + tx holds a(row = bi*32+tx, col = bj*32+ty+8q)
        const int src_r = bi * 32 + tx, src_c = bj * 32 + ty + 8 * q;
        if (src_r < n && src_c < n && src_r > src_c) W[(long)src_c * ldw + src_r] = t[tx][ty + 8 * q];
    }
}

// Wt[j][i] = W[i][j] (32 x 32 tiles through shared memory).
template <typename T>
__global__ void __launch_bounds__(256)
transpose_kernel(int n, const T *__restrict__ W, long ldw, T *__restrict__ Wt, long ldwt) {
    __shared__ T t[32][33];
    const int bi = blockIdx.y, bj = blockIdx.x;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int r = bi * 32 + ty + 8 * q, c = bj * 32 + tx;
        t[ty + 8 * q][tx] = (r < n && c < n) ? W[(long)r * ldw + c] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int r = bj * 32 + ty + 8 * q, c = bi * 32 + tx;  // Wt row r = W column r
        if (r < n && c < n) Wt[(long)r * ldwt + c] = t[tx][ty + 8 * q];
    }
}

}  // namespace

template <typename T>
cudaError_t launch_transpose(int n, const T *W, long ldw, T *Wt, long ldwt, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int nt = (n + 31) / 32;
    mp_note_launch();
    transpose_kernel<T><<<dim3(nt, nt), 256, 0, s>>>(n, W, ldw, Wt, ldwt);
    return cudaGetLastError();
}
template cudaError_t launch_transpose<float>(int, const float *, long, float *, long, cudaStream_t);
template cudaError_t launch_transpose<double>(int, const double *, long, double *, long, cudaStream_t);

int potrf_leaf_width() { return kLeaf; }

template <typename T>
cudaError_t launch_potrf_leaf(int n, int k0, int nc, T *W, long ldw, MpDevStatus *st, cudaStream_t s) {
    if (nc <= 0) return cudaSuccess;
    if (nc > kLeaf) return cudaErrorInvalidValue;
    const int below = n - k0 - nc;
    const int grid = below > 0 ? (below + kLeafRows - 1) / kLeafRows : 1;
    const size_t smem = sizeof(T) * kLeafRows * (kLeaf + 1);
    auto kern = potrf_leaf_kernel<T>;
    cudaError_t e = mp_smem_attr(kern, smem);
    if (e != cudaSuccess) return e;
    mp_note_launch();
    kern<<<grid, kLeafRows, smem, s>>>(n, k0, nc, W, ldw, st);
    return cudaGetLastError();
}
template cudaError_t launch_potrf_leaf<float>(int, int, int, float *, long, MpDevStatus *, cudaStream_t);
template cudaError_t launch_potrf_leaf<double>(int, int, int, double *, long, MpDevStatus *, cudaStream_t);

template <typename T>
cudaError_t launch_mirror_lower(int n, T *W, long ldw, cudaStream_t s) {
    if (n <= 1) return cudaSuccess;
    const int nt = (n + 31) / 32;
    mp_note_launch();
    mirror_lower_kernel<T><<<dim3(nt, nt), 256, 0, s>>>(n, W, ldw);
    return cudaGetLastError();
}
template cudaError_t launch_mirror_lower<float>(int, float *, long, cudaStream_t);
template cudaError_t launch_mirror_lower<double>(int, double *, long, cudaStream_t);
