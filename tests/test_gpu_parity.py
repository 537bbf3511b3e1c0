"""GPU parity: each step of the hot path and the whole solve, called through
the C ABI, against the CPU oracle on the same seeded inputs.

Tolerances (derived from the arithmetic, see the design notes):
  * conversion W = fl32(A): bit-exact (both sides round to nearest even);
  * pivots: bit-exact on pivot-unambiguous matrices; otherwise partial
    pivoting is checked by |l_ij| <= 1 (the chosen pivot dominated its column);
  * factors: ||PA - LU||_inf / ||A||_inf <= c n u_p;
  * residual: |r_gpu - r_exact| <= 2 n u64 (|A||x| + |b|) elementwise;
  * solve: every column bwd <= 1e-14 and ||x - x_oracle|| / ||x_oracle||
    <= 10 kappa_inf(A) 2^-53.
"""
import numpy as np
import pytest

from paper_0808_2794_gb300 import inputs

pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53
U32 = 2.0 ** -24
UP = {"fp32": U32, "fp16x3": U32, "bf16": 2.0 ** -8, "fp16": 2.0 ** -11}


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need a CUDA device"
    return t


@pytest.fixture(scope="module")
def mp():
    from paper_0808_2794_gb300 import solver
    solver.load()
    return solver


def dev(torch, a):
    """numpy (column-major or 1-D) -> CUDA tensor with the same column-major layout."""
    a = np.asarray(a)
    if a.ndim == 1:
        return torch.from_numpy(a.copy()).cuda()
    return torch.from_numpy(np.asfortranarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def unambiguous_matrix(n, seed):
    """A = P0^T L0 U0 with |l_ij| <= 1/(2 sqrt(n)): exact partial pivoting
    picks the rows of P0 with a margin of 2 sqrt(n) at every step.  L0 and U0
    (off-diagonal entries O(1/sqrt(n)), |u_ii| in [1, 2]) are well conditioned,
    so no rounding order can change a pivot decision."""
    rng = np.random.default_rng(seed)
    L0 = np.tril(rng.uniform(-0.5, 0.5, (n, n)) / np.sqrt(n), -1) + np.eye(n)
    U0 = (np.triu(rng.uniform(-1, 1, (n, n)), 1) / np.sqrt(n)
          + np.diag(rng.uniform(1, 2, n) * rng.choice([-1, 1], n)))
    perm = rng.permutation(n)
    A = np.empty((n, n))
    A[perm, :] = L0 @ U0  # row perm[i] of A is row i of L0 U0
    return np.asfortranarray(A)



# ------------------------------------------------------------ a1: conversion

@pytest.mark.parametrize("n", [1, 5, 33, 100, 257])
def test_convert_bitexact(torch, mp, orc, n):
    A, _, _ = inputs.dense_system(n, seed=n)
    A = np.asfortranarray(A * 10.0 ** np.random.default_rng(1).uniform(-3, 3, (n, n)))
    W, anorm, flags = mp.convert(dev(torch, A))
    W = host(W)[:, :n]
    assert np.array_equal(W, A.astype(np.float32))  # row-major W[i, j] = fl32(A[i, j])
    assert abs(host(anorm)[0] - orc.norm_inf(A)) <= 2 * n * U64 * orc.norm_inf(A)
    assert host(flags)[0] == 0
    A[n // 2, n // 3] = np.inf
    _, _, flags = mp.convert(dev(torch, A))
    assert host(flags)[0] & mp.FLAG_NONFINITE_INPUT


def _special_doubles(n, seed):
    """n x n FP64 values that reach every branch of round-to-nearest-even into
    binary32: uniformly random bit patterns (all exponents: overflow, the
    binary32 subnormal range, binary64 subnormals, infinities, NaNs), exact
    ties between adjacent binary32 values (normal and subnormal), the
    neighbours of every tie, the overflow threshold and signed zeros."""
    rng = np.random.default_rng(seed)
    bits = rng.integers(0, 2 ** 63, size=n * n, dtype=np.int64).astype(np.uint64)
    bits |= rng.integers(0, 2, size=n * n).astype(np.uint64) << np.uint64(63)
    v = bits.view(np.float64).copy()
    m = n * n // 2
    f = rng.standard_normal(m // 3).astype(np.float32) * np.float32(2.0) ** rng.integers(-140, 120, m // 3)
    f = np.where(np.isfinite(f) & (f != 0), f, np.float32(1.5))
    g = np.nextafter(f, np.float32(np.inf))
    tie = (f.astype(np.float64) + g.astype(np.float64)) / 2.0  # exact in binary64
    around = np.concatenate([tie, np.nextafter(tie, np.inf), np.nextafter(tie, -np.inf)])
    v[: around.size] = around
    fmax = float(np.finfo(np.float32).max)
    ulp = fmax - float(np.nextafter(np.float32(fmax), np.float32(0)))
    edge = [fmax, fmax + ulp / 2, np.nextafter(fmax + ulp / 2, 0), np.nextafter(fmax + ulp / 2, np.inf),
            2.0 ** -149, 2.0 ** -150, np.nextafter(2.0 ** -150, 1), 3 * 2.0 ** -151, 2.0 ** -126,
            np.nextafter(2.0 ** -126, 0), 0.0, -0.0, 5e-324, np.inf, -np.inf, np.nan]
    v[around.size: around.size + len(edge)] = edge
    v[around.size + len(edge): around.size + 2 * len(edge)] = -np.array(edge)
    return np.asfortranarray(v.reshape(n, n))


def test_convert_rounding_special_values(torch, mp):
    """fl32 of every class of binary64 value, bit for bit against the host's
    IEEE conversion (numpy, round to nearest even); NaN maps to NaN."""
    n = 96
    A = _special_doubles(n, seed=7)
    with np.errstate(over="ignore", invalid="ignore"):
        want = A.astype(np.float32)
    W, _, flags = mp.convert(dev(torch, A))
    W = host(W)[:, :n]
    nan = np.isnan(want)
    assert np.array_equal(np.isnan(W), nan)
    assert np.array_equal(W[~nan].view(np.uint32), want[~nan].view(np.uint32))
    assert host(flags)[0] & mp.FLAG_NONFINITE_INPUT


# ------------------------------------------------ a2-a4: panel, swaps, TRSM

def _factor(torch, mp, A, prec="fp32", nb_outer=0):
    W, _, _ = mp.convert(dev(torch, A))
    ipiv, info, flags = mp.getrf_lowp(W, prec=prec, nb_outer=nb_outer)
    torch.cuda.synchronize()
    n = A.shape[0]
    return W, host(W)[:, :n].astype(np.float64), host(ipiv), info, flags


def _check_factors(A, LU, piv, u, c=8.0):
    n = A.shape[0]
    L = np.tril(LU, -1) + np.eye(n)
    U = np.triu(LU)
    PA = A.copy()
    for k, p in enumerate(piv):
        PA[[k, p - 1], :] = PA[[p - 1, k], :]
    rel = np.max(np.sum(np.abs(PA - L @ U), axis=1)) / np.max(np.sum(np.abs(A), axis=1))
    assert rel <= c * n * u, rel
    assert np.all(np.abs(np.tril(LU, -1)) <= 1.0 + 4 * u)
    assert all(p >= k + 1 for k, p in enumerate(piv))
    return rel


@pytest.mark.parametrize("n", [1, 2, 3, 17, 31, 32, 33, 64, 65, 127, 129, 300, 513])
def test_getrf_fp32_pivots_exact(torch, mp, orc, n):
    A = unambiguous_matrix(n, seed=n)
    _, LU, piv, info, flags = _factor(torch, mp, A, nb_outer=64)
    LUo, pivo, infoo = orc.getrf(A, prec=32)
    assert info == 0 and flags == 0
    assert np.array_equal(piv, pivo)  # bit-exact index work
    _check_factors(A, LU, piv, U32)
    # with the pivots fixed, both factorizations are backward stable for the
    # same PA; their difference is bounded through the conditioning of L0, U0
    scale = np.max(np.abs(LUo))
    assert np.max(np.abs(LU - LUo.astype(np.float64))) <= 64 * n * U32 * scale


@pytest.mark.parametrize("n,nb", [(100, 32), (700, 128), (1024, 0), (2000, 256), (1500, 384), (2500, 448)])
def test_getrf_fp32_random_invariants(torch, mp, orc, n, nb):
    A, _, _ = inputs.dense_system(n, seed=n + 1)
    _, LU, piv, info, flags = _factor(torch, mp, A, nb_outer=nb)
    assert info == 0 and flags == 0
    _check_factors(A, LU, piv, U32, c=16.0)
    # pivots agree with the oracle up to the first column where the two
    # choices are a near tie: there the candidates' magnitudes in the FP64
    # Schur complement (under the oracle's earlier pivots) agree to rounding
    _, pivo, _ = orc.getrf(A, prec=32)
    _assert_pivots_until_near_tie(A, np.asarray(piv), np.asarray(pivo), tol=64 * n * U32)


def _assert_pivots_until_near_tie(A, piv, pivo, tol):
    diff = np.nonzero(piv != pivo)[0]
    if diff.size == 0:
        return
    j = int(diff[0])
    n = A.shape[0]
    perm = np.arange(n)
    for k in range(j):  # the oracle's row interchanges for columns 0 .. j-1
        q = pivo[k] - 1
        perm[[k, q]] = perm[[q, k]]
    PA = A[perm]
    s = PA[j:, j] - PA[j:, :j] @ np.linalg.solve(PA[:j, :j], PA[:j, j]) if j > 0 else PA[j:, j]
    a_gpu, a_orc = abs(s[piv[j] - 1 - j]), abs(s[pivo[j] - 1 - j])
    assert abs(a_gpu - a_orc) <= tol * max(a_gpu, a_orc), (j, a_gpu, a_orc)


def test_getrf_zero_pivot_reports_info(torch, mp):
    n = 40
    A = np.asfortranarray(np.random.default_rng(3).standard_normal((n, n)))
    A[:, 7] = 0.0  # a zero column: the first zero pivot is column 8 (1-based)
    _, _, piv, info, flags = _factor(torch, mp, A)
    assert info == 8 and flags & mp.FLAG_LOWP_BREAKDOWN


# --------------------------------------------------- a5: trailing update GEMM

@pytest.mark.parametrize("prec", ["fp32", "fp16x3", "bf16", "fp16"])
@pytest.mark.parametrize("M,N,K", [(256, 128, 64), (300, 200, 100), (1000, 777, 512), (129, 1025, 33)])
def test_trailing_update(torch, mp, orc, prec, M, N, K):
    rng = np.random.default_rng(M + N + K)
    ld = lambda c: (c + 3) // 4 * 4
    L = rng.uniform(-1, 1, (M, K))
    U = rng.standard_normal((K, N)) * 3
    C = rng.standard_normal((M, N))
    Lt = torch.zeros((M, ld(K)), dtype=torch.float32, device="cuda")
    Ut = torch.zeros((K, ld(N)), dtype=torch.float32, device="cuda")
    Ct = torch.zeros((M, ld(N)), dtype=torch.float32, device="cuda")
    Lt[:, :K] = torch.from_numpy(L.astype(np.float32)).cuda()
    Ut[:, :N] = torch.from_numpy(U.astype(np.float32)).cuda()
    Ct[:, :N] = torch.from_numpy(C.astype(np.float32)).cuda()
    mp.lowp_gemm_update(Ct[:, :N], Lt[:, :K], Ut[:, :N], prec=prec)
    got = host(Ct)[:, :N].astype(np.float64)
    L32, U32_, C32 = (x.astype(np.float32).astype(np.float64) for x in (L, U, C))
    if prec in ("bf16", "fp16"):
        L32 = orc.round_to(L32, prec)
        U32_ = orc.round_to(U32_, prec)
    ref = C32 - L32 @ U32_  # FP64: products of the rounded operands are exact
    # fp16x3: each operand is hi + lo to about 2^-22 (relative) plus the fp16
    # subnormal quantum after power-of-two scaling; the dropped lo*lo term is
    # below 2^-22 -- a few extra units of u32 per product
    extra = 24 if prec == "fp16x3" else 2
    bound = (K + extra) * U32 * (np.abs(L32) @ np.abs(U32_) + np.abs(C32))
    assert np.all(np.abs(got - ref) <= bound)


# ------------------------------------------------ a7: triangular solves

@pytest.mark.parametrize("n,nrhs", [(1, 1), (63, 1), (64, 2), (65, 1), (200, 3), (1000, 1), (1500, 8)])
def test_getrs_against_fp64_substitution(torch, mp, orc, n, nrhs):
    A, _, _ = inputs.dense_system(n, seed=2 * n)
    A = np.asfortranarray(A + np.sqrt(n) * np.eye(n))  # keep L, U well conditioned
    W, LU, piv, info, _ = _factor(torch, mp, A)
    rng = np.random.default_rng(n)
    R = np.asfortranarray(rng.standard_normal((n, nrhs)) * 1e-9)
    Z = host(mp.getrs_lowp(W, torch.from_numpy(piv).cuda(), dev(torch, R)))
    Zref = orc.getrs(LU, piv, R, prec=64)  # same FP32 factors, FP64 substitution
    rel = np.max(np.abs(Z - Zref)) / np.max(np.abs(Zref))
    assert rel <= 64 * n * U32, rel


# ------------------------------------------------------- a8: FP64 residual

@pytest.mark.parametrize("n,nrhs", [(1, 1), (7, 2), (256, 1), (1000, 4), (3001, 8)])
def test_residual_fp64(torch, mp, orc, n, nrhs):
    A, B, X = inputs.dense_system(n, nrhs=nrhs, seed=n)
    X = X + np.random.default_rng(0).standard_normal(X.shape) * 1e-10
    R = host(mp.residual(dev(torch, A), dev(torch, X), dev(torch, B)))
    Rex = orc.residual(A, X, B, compensated=True)
    bound = 2 * n * U64 * (np.abs(A) @ np.abs(X) + np.abs(B))
    assert np.all(np.abs(R - Rex) <= bound)


# ---------------------------------------------------- whole solve (Alg. 1)

def _check_solution(orc, A, B, X, kappa=None):
    bwd = orc.bwd_err(A, X, B)
    assert np.all(bwd <= 1e-14), bwd
    ref = orc.gesv_ir(A, B, factor_prec=64)["X"]
    ref = ref.reshape(X.shape)
    kappa = orc.kappa_inf(A) if kappa is None else kappa
    fwd = np.max(np.abs(X - ref)) / np.max(np.abs(ref))
    assert fwd <= 10 * kappa * U64, (fwd, kappa)


@pytest.mark.parametrize("n,nrhs", [(1, 1), (2, 1), (3, 2), (17, 1), (64, 1), (100, 3), (127, 1),
                                    (129, 2), (257, 1), (1024, 1)])
def test_gesv_fp32(torch, mp, orc, n, nrhs):
    A, B, _ = inputs.dense_system(n, nrhs=nrhs, seed=n)
    X, piv, st = mp.gesv(dev(torch, A), dev(torch, B), prec="fp32")
    X = host(X)
    assert st["flags"] == 0 and st["iter"] >= 0, st
    _check_solution(orc, A, B, X)
    # sanity bound on the work: the GPU solves with inverted diagonal blocks
    # (different rounding from substitution), so its contraction per
    # correction can be somewhat weaker than the oracle's
    r = orc.gesv_ir(A, B, factor_prec=32)
    assert st["iter"] <= 2 * r["iter"] + 3


def test_gesv_identity_and_permutation(torch, mp):
    n = 50
    b = np.arange(1.0, n + 1)
    X, piv, st = mp.gesv(dev(torch, np.eye(n, order="F")), dev(torch, b))
    assert st["iter"] == 0 and np.array_equal(host(X), b)
    perm = np.random.default_rng(5).permutation(n)
    P = np.zeros((n, n), order="F")
    P[np.arange(n), perm] = 1.0
    X, piv, st = mp.gesv(dev(torch, P), dev(torch, b))
    assert st["iter"] == 0 and np.array_equal(host(X), P.T @ b)


def test_gesv_hilbert_falls_back(torch, mp, orc):
    n = 10
    H = np.array([[1.0 / (i + j + 1) for j in range(n)] for i in range(n)], order="F")
    b = np.ones(n)
    X, piv, st = mp.gesv(dev(torch, H), dev(torch, b))
    assert st["flags"] & mp.FLAG_FALLBACK and st["iter"] == -1
    assert orc.bwd_err(H, host(X), b)[0] <= 1e-14


def test_gesv_itermax_zero_forces_fallback(torch, mp, orc):
    A, B, _ = inputs.dense_system(80, seed=9)
    X, piv, st = mp.gesv(dev(torch, A), dev(torch, B), itermax=0)
    assert st["flags"] & mp.FLAG_FALLBACK
    assert np.all(orc.bwd_err(A, host(X), B) <= 1e-14)
    X, piv, st = mp.gesv(dev(torch, A), dev(torch, B), itermax=0, allow_fallback=False)
    assert st["flags"] & mp.FLAG_NOT_CONVERGED


def test_gesv_fp64_fallback_factorization(torch, mp, orc):
    """itermax = 0 forces the FP64 fallback: the FP64 LU runs through the same
    leaf pipeline as the low-precision one (panel kernel applying the previous
    leaf on load, bulk launches with the left-looking U rows), here over
    several 128-wide outer panels with a ragged last one.  The FP64 solve is
    compared with the oracle's FP64 solve."""
    n = 1000
    A, B, _ = inputs.dense_system(n, nrhs=2, seed=12)
    X, piv, st = mp.gesv(dev(torch, A), dev(torch, B), itermax=0, nb_outer=128)
    assert st["flags"] & mp.FLAG_FALLBACK
    X = host(X).reshape(n, 2)
    assert np.all(orc.bwd_err(A, X, B) <= 1e-14)
    ref = orc.gesv_ir(A, B, factor_prec=64)["X"].reshape(n, 2)
    assert np.max(np.abs(X - ref)) / np.max(np.abs(ref)) <= 10 * orc.kappa_inf(A) * U64


def test_gesv_singular_reports_info(torch, mp):
    n = 30
    A = np.asfortranarray(np.random.default_rng(1).standard_normal((n, n)))
    A[:, 4] = 0.0
    X, piv, st = mp.gesv(dev(torch, A), dev(torch, np.ones(n)))
    assert st["info_fp64"] == 5 and st["flags"] & mp.FLAG_FALLBACK


def test_gesv_nonfinite_input(torch, mp):
    A, B, _ = inputs.dense_system(20, seed=1)
    A = A.copy(order="F")
    A[3, 3] = np.nan
    X, piv, st = mp.gesv(dev(torch, A), dev(torch, B))
    assert st["flags"] & mp.FLAG_NONFINITE_INPUT


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
@pytest.mark.parametrize("n", [300, 1100, 2048])
def test_gesv_lowp_tensor_cores(torch, mp, orc, prec, n):
    A, B, _ = inputs.dense_system(n, seed=n)
    A = np.asfortranarray(A + 2 * np.sqrt(n) * np.eye(n))  # kappa small enough for classical IR
    X, piv, st = mp.gesv(dev(torch, A), dev(torch, B), prec=prec, nb_outer=128)
    assert not st["flags"] & mp.FLAG_FALLBACK, st
    _check_solution(orc, A, B, host(X))


@pytest.mark.parametrize("n", [300, 1100, 2048])
def test_gesv_fp16x3_plain_dense(torch, mp, orc, n):
    """The split-fp16 rung is as accurate as the FP32 factorization: classical
    refinement converges on plain N(0,1) systems with no fallback."""
    A, B, _ = inputs.dense_system(n, nrhs=2, seed=n + 5)
    X, piv, st = mp.gesv(dev(torch, A), dev(torch, B), prec="fp16x3", nb_outer=256)
    assert st["flags"] == 0, st
    _check_solution(orc, A, B, host(X))
    r = orc.gesv_ir(A, B, factor_prec=32)
    assert st["iter"] <= 2 * r["iter"] + 3


@pytest.mark.parametrize("prec", ["bf16", "fp16", "fp16x3"])
def test_getrf_lowp_factor_bound(torch, mp, orc, prec):
    n = 1500
    A, _, _ = inputs.dense_system(n, seed=7)
    _, LU, piv, info, flags = _factor(torch, mp, A, prec=prec, nb_outer=256)
    assert info == 0
    _check_factors(A, LU, piv, UP[prec], c=4.0)


def test_gesv_host_entry_point(torch, mp, orc):
    A, B, _ = inputs.dense_system(600, nrhs=2, seed=4)
    X, piv, st = mp.gesv_host(A, B)
    assert st["flags"] == 0
    _check_solution(orc, A, B, X)
