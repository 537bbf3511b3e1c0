"""Pins for the CPU oracle: exact rationals, closed forms, invariants, special
cases and library special cases.  None of these re-types the oracle's own
formula; each compares it with something the mathematics fixes.

Runs on CPU (no GPU marker).
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import exact
from paper_0808_2794_gb300 import inputs

U64 = 2.0 ** -53
U32 = 2.0 ** -24


def _exact_has_pivot_tie(A):
    """True if exact GEPP meets a tie (or near-tie) in a pivot choice."""
    n = len(A)
    M = [row[:] for row in A]
    for k in range(n):
        mags = sorted((abs(M[i][k]) for i in range(k, n)), reverse=True)
        if len(mags) > 1 and mags[0] != 0 and (mags[0] - mags[1]) <= mags[0] * Fraction(1, 1000):
            return True
        p = max(range(k, n), key=lambda i: (abs(M[i][k]), -i))
        if M[p][k] == 0:
            return True
        M[k], M[p] = M[p], M[k]
        for i in range(k + 1, n):
            M[i][k] = M[i][k] / M[k][k]
            for j in range(k + 1, n):
                M[i][j] -= M[i][k] * M[k][j]
    return False


# ---------------------------------------------------------------- LU (Sec. 2.1)

@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
@pytest.mark.parametrize("seed", range(6))
def test_getrf_matches_exact_gepp(orc, n, seed):
    A = inputs.small_integer_matrix(n, seed=100 * n + seed)
    Af = exact.to_frac_matrix(A.tolist())
    if _exact_has_pivot_tie(Af):
        pytest.skip("pivot choice not unique at this tolerance")
    L, U, ipiv, info = exact.gepp(Af)
    for prec, u in ((64, U64), (32, U32)):
        LU, piv, inf = orc.getrf(A, prec=prec)
        assert inf == info == 0
        assert list(piv) == ipiv, (prec, list(piv), ipiv)
        scale = max(float(abs(v)) for row in U for v in row)
        for i in range(n):
            for j in range(n):
                ref = float(L[i][j]) if j < i else float(U[i][j])
                assert abs(LU[i, j] - ref) <= 64 * n * u * max(scale, 1.0), (prec, i, j)


def test_getrf_tie_goes_to_smallest_index(orc):
    # column 0 holds 3, -3, 3: exact tie, the smallest row index must win (no swap)
    A = np.array([[3.0, 1, 2], [-3.0, 5, 1], [3.0, 2, 7]], order="F")
    for prec in (64, 32):
        _, piv, _ = orc.getrf(A, prec=prec)
        assert piv[0] == 1
    B = np.array([[1.0, 1, 2], [-3.0, 5, 1], [3.0, 2, 7]], order="F")
    for prec in (64, 32):
        _, piv, _ = orc.getrf(B, prec=prec)
        assert piv[0] == 2  # rows 2 and 3 tie at |3|: row 2 (1-based) wins
    L, U, ip, _ = exact.gepp(exact.to_frac_matrix(B.tolist()))
    assert ip[0] == 2


@pytest.mark.parametrize("n", [2, 4, 7])
def test_getrs_matches_exact_solve(orc, n):
    A = inputs.small_integer_matrix(n, seed=7 + n)
    A[np.diag_indices(n)] += 20.0  # well conditioned, nonsingular
    b = np.arange(1, n + 1, dtype=np.float64)
    x_ex = exact.solve(exact.to_frac_matrix(A.tolist()), [Fraction(v) for v in b])
    LU, piv, info = orc.getrf(A)
    x = orc.getrs(LU, piv, b)
    kappa = orc.kappa_inf(A)
    for i in range(n):
        assert abs(x[i] - float(x_ex[i])) <= 10 * kappa * U64 * max(abs(float(v)) for v in x_ex)


@pytest.mark.parametrize("n", [2, 3, 5, 8])
@pytest.mark.parametrize("seed", range(4))
def test_getrs_trans_matches_exact_transposed_solve(orc, n, seed):
    """A^T x = b solved with the LU factors of A (U^T L^T P x = b: U^T forward,
    L^T backward, then the row exchanges undone in reverse order) against the
    exact rational solve of the transposed system.  The diagonal of A is zeroed
    so that partial pivoting must exchange rows; several exchanges that do not
    commute make the order of the final permutation visible."""
    A = inputs.small_integer_matrix(n, seed=300 + 10 * n + seed, lo=-99, hi=99)
    A[np.diag_indices(n)] = 0.0
    Af = exact.to_frac_matrix(A.tolist())
    if _exact_has_pivot_tie(Af):
        pytest.skip("pivot choice not unique at this tolerance")
    At = [[Af[j][i] for j in range(n)] for i in range(n)]
    b = np.array([(-1.0) ** i * (i + 2) for i in range(n)])
    x_ex = exact.solve(At, [Fraction(v) for v in b])
    kappa = float(exact.norm_inf(At) * exact.norm_inf(exact.inverse(At)))
    LU, piv, info = orc.getrf(A)
    assert info == 0
    assert any(p != k + 1 for k, p in enumerate(piv))
    x = orc.getrs_trans(LU, piv, b)
    xm = max(abs(float(v)) for v in x_ex)
    for i in range(n):
        assert abs(x[i] - float(x_ex[i])) <= 10 * kappa * U64 * xm, (i, x[i], float(x_ex[i]))
    # several right-hand sides are independent columns
    B2 = np.stack([b, -2.0 * b[::-1]], axis=1)
    X2 = orc.getrs_trans(LU, piv, B2)
    x2_ex = exact.solve(At, [Fraction(v) for v in B2[:, 1]])
    assert np.array_equal(X2[:, 0], x)
    for i in range(n):
        assert abs(X2[i, 1] - float(x2_ex[i])) <= 10 * kappa * U64 * max(abs(float(v)) for v in x2_ex)


@pytest.mark.parametrize("n", [3, 6, 8])
def test_matvec_dot2_against_exact(orc, n):
    """b = A x with the compensated Dot2 product is the exact rational A x
    rounded once, up to the Dot2 bound, on products that cancel almost
    completely (the last column of A is chosen so that A x is tiny next to
    |A| |x|, where a plain FP64 sum would be wrong in most digits)."""
    rng = np.random.default_rng(1000 + n)
    A = rng.standard_normal((n, 2 * n))[:, :n].copy(order="F")
    X = rng.standard_normal((n, 2))
    A[:, -1] = -(A[:, :-1] @ X[:-1, 0]) / X[-1, 0] + rng.standard_normal(n) * 1e-13
    B = orc.matvec_dot2(A, X)
    Af = exact.to_frac_matrix(A.tolist())
    absterm = np.abs(A) @ np.abs(X)
    for c in range(2):
        xc = [Fraction(v) for v in X[:, c]]
        for i in range(n):
            e = float(sum(Af[i][j] * xc[j] for j in range(n)))
            assert abs(B[i, c] - e) <= U64 * abs(e) + 4 * (n + 1) ** 2 * U64 ** 2 * absterm[i, c], (c, i)
    # the cancelling column is the one that separates Dot2 from a plain sum
    assert np.max(np.abs(B[:, 0]) / absterm[:, 0]) < 1e-9
    b1 = orc.matvec_dot2(A, X[:, 1])
    assert b1.shape == (n,) and np.array_equal(b1, B[:, 1])


@pytest.mark.parametrize("n", [3, 5, 8])
@pytest.mark.parametrize("seed", range(4))
def test_refined_solution_matches_exact_solve(orc, n, seed):
    """Algorithm 1 with an FP32 factor, run to the FP64 floor, gives the exact
    solution to within 10 kappa_inf u64 (forward error) and bwd <= 1e-14."""
    A = inputs.small_integer_matrix(n, seed=50 + 10 * n + seed)
    A[np.diag_indices(n)] += 10.0
    Af = exact.to_frac_matrix(A.tolist())
    b = np.arange(1.0, n + 1) * (-1) ** np.arange(n)
    x_ex = np.array([float(v) for v in exact.solve(Af, [Fraction(v) for v in b])])
    inv = exact.inverse(Af)
    kappa = float(exact.norm_inf(Af) * exact.norm_inf(inv))
    r = orc.gesv_ir(A, b, factor_prec=32)
    assert r["flags"] == 0 and r["bwd"] <= 1e-14
    assert np.max(np.abs(r["X"] - x_ex)) <= 10 * kappa * U64 * np.max(np.abs(x_ex))


def test_singular_matrix_reports_info(orc):
    A = inputs.small_integer_matrix(6, seed=3)
    A[4, :] = A[1, :]  # duplicate rows
    _, _, info = orc.getrf(A)
    assert info > 0
    Af = exact.to_frac_matrix(A.tolist())
    assert exact.gepp(Af)[3] > 0
    r = orc.gesv_ir(A, np.ones(6), factor_prec=64)
    assert r["info"] > 0


def test_tridiagonal_closed_form(orc):
    n = 50
    T = np.asfortranarray(2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1))
    ukk, lsub = exact.tridiag_lu_closed_form(n)
    for prec, u in ((64, U64), (32, U32)):
        LU, piv, info = orc.getrf(T, prec=prec)
        assert info == 0 and list(piv) == list(range(1, n + 1))  # no exchanges
        for k in range(n):
            assert abs(LU[k, k] - float(ukk[k])) <= 4 * n * u
        for k in range(n - 1):
            assert abs(LU[k + 1, k] - float(lsub[k])) <= 4 * n * u
            assert LU[k, k + 1] == -1.0
    # kappa_inf from the closed-form inverse
    inv = exact.tridiag_inverse_closed_form(n)
    kap = 4 * max(sum(abs(v) for v in row) for row in inv)
    assert abs(orc.kappa_inf(T) - float(kap)) <= 1e-10 * float(kap)
    # b = T x_true exact in small integers -> refinement recovers x_true
    x_true = np.arange(-n // 2, n - n // 2, dtype=np.float64)
    b = T @ x_true  # exact: small integers
    r = orc.gesv_ir(T, b, factor_prec=32)
    assert r["flags"] == 0 and r["bwd"] <= 1e-14
    assert np.max(np.abs(r["X"] - x_true)) <= 10 * orc.kappa_inf(T) * U64 * np.max(np.abs(x_true))


def test_hilbert_closed_form_and_fallback(orc):
    for n in (4, 6, 8):
        H = np.array([[1.0 / (i + j + 1) for j in range(n)] for i in range(n)], order="F")
        inv = exact.hilbert_inverse_closed_form(n)
        kap_exact = float(exact.norm_inf(exact.hilbert(n)) * exact.norm_inf(inv))
        # the FP64 H differs from the exact H by rounding: relative kappa
        # perturbation is about kappa * u
        assert abs(orc.kappa_inf(H) - kap_exact) <= 100 * kap_exact ** 2 * U64 + 1e-12 * kap_exact
    # n = 8: kappa ~ 3e10 > 1/u32 -> single-precision refinement cannot
    # converge (Section 4), the oracle resorts to FP64
    H8 = np.array([[1.0 / (i + j + 1) for j in range(8)] for i in range(8)], order="F")
    r = orc.gesv_ir(H8, np.ones(8), factor_prec=32)
    assert r["flags"] & orc.FALLBACK and r["iter"] == -1
    assert r["bwd"] <= 1e-14


def test_lu_invariants_random(orc):
    for n in (37, 100):
        A, _, _ = inputs.dense_system(n, seed=n)
        for prec, u in ((64, U64), (32, U32)):
            LU, piv, info = orc.getrf(A, prec=prec)
            LU = LU.astype(np.float64)
            L = np.tril(LU, -1) + np.eye(n)
            U = np.triu(LU)
            PA = A.copy()
            for k, p in enumerate(piv):
                PA[[k, p - 1], :] = PA[[p - 1, k], :]
            rel = np.max(np.sum(np.abs(PA - L @ U), axis=1)) / orc.norm_inf(A)
            assert rel <= 2 * n * u * 10  # c*n*u with modest growth allowance
            assert np.all(np.abs(np.tril(LU, -1)) <= 1.0)
            assert all(p >= k + 1 for k, p in enumerate(piv))


def test_permutation_and_diagonal_special_cases(orc):
    n = 9
    perm = np.random.default_rng(5).permutation(n)
    P = np.zeros((n, n), order="F")
    P[np.arange(n), perm] = 1.0
    b = np.arange(1.0, n + 1)
    r = orc.gesv_ir(P, b, factor_prec=32)
    assert r["iter"] == 0 and r["flags"] == 0
    assert np.array_equal(r["X"], P.T @ b)
    D = np.asfortranarray(np.diag(np.arange(1.0, n + 1)))
    _, piv, _ = orc.getrf(D)
    assert list(piv) == list(range(1, n + 1))
    r = orc.gesv_ir(np.eye(n, order="F"), b, factor_prec=32)
    assert r["iter"] == 0 and np.array_equal(r["X"], b)


# ------------------------------------------------------- residual (Alg. 1 step 4)

@pytest.mark.parametrize("n", [3, 6, 8])
def test_residual_against_exact(orc, n):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n))
    x = rng.standard_normal(n)
    b = A @ x + rng.standard_normal(n) * 1e-12  # tiny residual: heavy cancellation
    Af = exact.to_frac_matrix(A.tolist())
    r_ex = exact.residual(Af, [Fraction(v) for v in x], [Fraction(v) for v in b])
    absterm = np.abs(b) + np.abs(A) @ np.abs(x)
    r2 = orc.residual(A, x, b, compensated=True)
    r1 = orc.residual(A, x, b, compensated=False)
    for i in range(n):
        e = float(r_ex[i])
        # Dot2: as if computed in twice the precision, then rounded once
        assert abs(r2[i] - e) <= U64 * abs(e) + 4 * (n + 1) ** 2 * U64 ** 2 * absterm[i]
        # plain FP64 sum: gamma_n bound
        assert abs(r1[i] - e) <= (n + 1) * U64 * absterm[i] * 1.01
    assert orc.norm_inf(A) == float(exact.norm_inf(exact.to_frac_matrix(np.abs(A).tolist())))


def test_bwd_err_definition(orc):
    n = 5
    A = inputs.small_integer_matrix(n, seed=11)
    x = np.array([1.0, -2.0, 0.5, 3.0, -1.0])
    b = A @ x  # exact
    assert np.all(orc.bwd_err(A, x, b) == 0.0)
    xp = x + np.array([0, 0, 0.25, 0, 0])
    r = b - A @ xp  # exact in binary
    want = np.max(np.abs(r)) / (orc.norm_inf(A) * np.max(np.abs(xp)) + np.max(np.abs(b)))
    assert orc.bwd_err(A, xp, b)[0] == pytest.approx(want, rel=1e-15)


# ------------------------------------------------------ Cholesky (Sec. 3.1.1)

def test_cholesky_against_exact_ldlt(orc):
    n = 6
    G = inputs.small_integer_matrix(n, seed=2)
    S = np.asfortranarray(G.T @ G + n * np.eye(n))
    L, D = exact.cholesky(exact.to_frac_matrix(S.tolist()))
    Lc = np.array([[float(L[i][j]) * np.sqrt(float(D[j])) for j in range(n)] for i in range(n)])
    for prec, u in ((64, U64), (32, U32)):
        F, info = orc.potrf(S, prec=prec)
        assert info == 0
        got = np.tril(F.astype(np.float64))
        assert np.max(np.abs(got - Lc)) <= 64 * n * u * np.max(np.abs(Lc))
    T = np.asfortranarray(2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1))
    F, info = orc.potrf(T)
    for k in range(n):
        assert abs(F[k, k] - np.sqrt((k + 2) / (k + 1))) <= 8 * U64
    N = S.copy(order="F")
    N[2, 2] = -50.0
    assert orc.potrf(N)[1] > 0


def test_posv_ir_spd(orc):
    A, B, X = inputs.conditioned_system(64, 1e3, nrhs=2, spd=True, seed=1)
    r = orc.posv_ir(A, B)
    assert r["flags"] == 0 and r["bwd"] <= 1e-14 and r["iter"] >= 1
    assert np.max(np.abs(r["X"] - X)) <= 10 * orc.kappa_inf(A) * U64 * 2


# ------------------------------------------- refinement behaviour (Sec. 4)

def test_iteration_count_against_datta_prediction(orc):
    """Section 4: ceil(ln eps_d / (ln eps_s + ln kappa)) iterations, valid while
    kappa*eps_s < 1.  The formula is stated for reaching the accuracy of the
    double-precision solve; with the (weaker) normwise backward-error stop the
    count must not exceed it, must be at least one correction, and must not
    decrease as kappa grows."""
    means = []
    for kappa in (1e1, 1e3, 1e5, 1e6):
        pred = int(np.ceil(np.log(U64) / (np.log(U32) + np.log(kappa))))
        its = []
        for seed in range(4):
            A, B, _ = inputs.conditioned_system(200, kappa, seed=seed)
            r = orc.gesv_ir(A, B[:, 0], factor_prec=32)
            assert r["flags"] == 0 and r["bwd"] <= 1e-14
            its.append(r["iter"])
        assert 1 <= np.mean(its) <= pred + 1, (kappa, its, pred)
        means.append(np.mean(its))
    assert all(a <= b for a, b in zip(means, means[1:])), means


def test_no_convergence_when_kappa_eps_s_above_one(orc):
    A, B, _ = inputs.conditioned_system(200, 1e9, seed=0)
    r = orc.gesv_ir(A, B[:, 0], factor_prec=32, allow_fallback=False)
    assert r["flags"] & (orc.STALLED | orc.BREAKDOWN) or r["iter"] == 30
    assert r["bwd"] > 1e-14
    r = orc.gesv_ir(A, B[:, 0], factor_prec=32)
    assert r["flags"] & orc.FALLBACK and r["bwd"] <= 1e-14


def test_itermax_zero_forces_fallback(orc):
    A, B, _ = inputs.dense_system(40, seed=3)
    r = orc.gesv_ir(A, B, factor_prec=32, itermax=0)
    assert r["flags"] & orc.FALLBACK and r["bwd"] <= 1e-14


def test_nonfinite_input_flag(orc):
    A, B, _ = inputs.dense_system(10, seed=4)
    A = A.copy(order="F")
    A[3, 3] = np.nan
    r = orc.gesv_ir(A, B, factor_prec=32, allow_fallback=False)
    assert r["flags"] & orc.NONFINITE


def test_multiple_rhs_equal_separate_solves(orc):
    A, B, _ = inputs.dense_system(60, nrhs=4, seed=8)
    r = orc.gesv_ir(A, B, factor_prec=32)
    for c in range(4):
        rc = orc.gesv_ir(A, B[:, c], factor_prec=32)
        assert np.max(np.abs(rc["X"] - r["X"][:, c])) <= 1e-13 * np.max(np.abs(rc["X"]))


def test_gmres_ir_recovers_beyond_classical(orc):
    """kappa*u32 > 1: classical single-precision refinement fails, while FGMRES
    preconditioned by the single-precision LU reaches FP64 backward error
    (Section 4, Arioli-Duff)."""
    A, B, X = inputs.conditioned_system(120, 1e8, seed=2)
    g = orc.gmres_ir(A, B[:, 0])
    assert g["outer"] >= 1 and g["bwd"] <= 1e-14
    I = np.eye(16, order="F")
    g = orc.gmres_ir(I, np.arange(16.0))
    assert g["outer"] == 0 and g["nmatvec"] == 0


def test_kappa_estimator_lower_bound(orc):
    for seed in range(3):
        A, _, _ = inputs.dense_system(80, seed=seed)
        k_true = np.linalg.cond(A, 1)
        k_est = orc.kappa_1_est(A)
        assert k_est <= k_true * (1 + 1e-10)
        assert k_est >= k_true / 10


def test_kappa_inf_estimator_from_lu_factors(orc):
    """The estimate of kappa_inf(A) = ||A||inf ||A^{-1}||inf taken from the
    LU factors of A (solves with A^T and A in swapped roles) is a lower bound
    within 10x of the exact value, on dense random matrices and on the
    tridiagonal Toeplitz matrix, whose inverse is known in closed form; on a
    non-symmetric matrix it differs from the 1-norm estimate."""
    for seed in range(3):
        A, _, _ = inputs.dense_system(80, seed=seed)
        LU, piv, info = orc.getrf(A)
        k_true = np.linalg.cond(A, np.inf)
        k_est = orc.kappa_inf_est_lu(A, LU, piv)
        assert k_true / 10 <= k_est <= k_true * (1 + 1e-10)
    n = 40
    T = np.asfortranarray(2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1))
    inv = exact.tridiag_inverse_closed_form(n)
    k_exact = 4.0 * float(exact.norm_inf(inv))
    LU, piv, _ = orc.getrf(T)
    k_est = orc.kappa_inf_est_lu(T, LU, piv)
    assert k_exact / 10 <= k_est <= k_exact * (1 + 1e-10)
    # a matrix whose 1-norm and inf-norm condition numbers differ widely
    A = np.asfortranarray(np.eye(30) + np.outer(np.r_[1e3, np.zeros(29)], np.ones(30)))
    LU, piv, _ = orc.getrf(A)
    k_inf = np.linalg.cond(A, np.inf)
    assert k_inf / 10 <= orc.kappa_inf_est_lu(A, LU, piv) <= k_inf * (1 + 1e-10)
    assert abs(np.linalg.cond(A, 1) - k_inf) > 0.5 * k_inf


# ------------------------------------------------------- rounding helpers

def _brute_nearest(x, grid):
    """Nearest grid value; ties to the one with even significand code."""
    i = np.searchsorted(grid[:, 0], x)
    cands = [grid[j] for j in (i - 1, i) if 0 <= j < len(grid)]
    best = min(cands, key=lambda g: (abs(g[0] - x), g[1] % 2))
    return best[0]


def test_round_fp16_matches_numpy(orc):
    rng = np.random.default_rng(0)
    xs = np.concatenate([rng.standard_normal(2000) * 10.0 ** rng.integers(-9, 5, 2000),
                         [65504.0, 65519.99, 65520.0, 2.0 ** -24, 2.0 ** -25, 3 * 2.0 ** -26]])
    got = orc.round_to(xs, "fp16")
    want = xs.astype(np.float16).astype(np.float64)
    assert np.array_equal(got, want)


def test_round_bf16_brute_force(orc):
    codes = np.arange(0, 0x7F80, dtype=np.uint32)  # positive finite bf16
    vals = (codes << 16).view(np.float32).astype(np.float64)
    grid = np.stack([vals, (codes & 0xFFFF).astype(np.float64)], axis=1)
    rng = np.random.default_rng(1)
    xs = np.abs(rng.standard_normal(3000) * 10.0 ** rng.integers(-30, 30, 3000))
    mids = (vals[1000:1010] + vals[1001:1011]) / 2  # exact ties
    for x in np.concatenate([xs, mids]):
        assert orc.round_to([x], "bf16")[0] == _brute_nearest(x, grid)
        assert orc.round_to([-x], "bf16")[0] == -_brute_nearest(x, grid)


def test_round_e4m3_brute_force(orc):
    # OCP E4M3: 1 sign, 4 exponent (bias 7), 3 mantissa; S.1111.111 is NaN; max 448
    vals = []
    for code in range(0, 0x7F):
        e, m = code >> 3, code & 7
        v = (m / 8.0) * 2.0 ** -6 if e == 0 else (1 + m / 8.0) * 2.0 ** (e - 7)
        vals.append((v, code))
    grid = np.array(sorted(vals))
    assert grid[-1, 0] == 448.0
    rng = np.random.default_rng(2)
    xs = np.abs(rng.standard_normal(2000) * 10.0 ** rng.integers(-4, 3, 2000))
    for x in xs:
        want = 448.0 if x > 448.0 else _brute_nearest(x, grid)
        assert orc.round_to([x], "e4m3")[0] == want


# ----------------------------------- extra-precise refinement (Section 5)

UDD = 2.0 ** -104


def _dd_frac(xh, xl):
    return [Fraction(float(h)) + Fraction(float(l)) for h, l in zip(xh, xl)]


@pytest.mark.parametrize("n", [2, 5, 8])
@pytest.mark.parametrize("seed", range(3))
def test_gesv_dd_matches_exact_solve(orc, n, seed):
    """FP64 factors, double-double residual and solution: the result
    Xhi + Xlo equals the exact rational solution to within the double-double
    level kappa u_dd (far below FP64's kappa u64)."""
    A = inputs.small_integer_matrix(n, seed=500 + 10 * n + seed, lo=-99, hi=99)
    A[np.diag_indices(n)] += 150.0
    b = np.array([1.0 / 3.0 + i for i in range(n)])  # not exactly representable in binary
    Af = exact.to_frac_matrix(A.tolist())
    x_ex = exact.solve(Af, [Fraction(v) for v in b])
    kappa = float(exact.norm_inf(Af) * exact.norm_inf(exact.inverse(Af)))
    r = orc.gesv_dd(A, b)
    assert r["info"] == 0 and r["iter"] >= 1
    x = _dd_frac(r["Xhi"], r["Xlo"])
    xm = max(abs(v) for v in x_ex)
    err = max(abs(a - e) for a, e in zip(x, x_ex))
    assert err <= 64 * n * kappa * UDD * xm, (float(err), float(xm))


def test_gesv_dd_on_floating_point_hilbert_matrix(orc):
    """The FP64 Hilbert matrix of order 10 (kappa ~ 1.6e13): the FP64 solve
    alone keeps about three digits; refinement with the double-double
    residual reaches the exact rational solution of that matrix to well
    below FP64's unit roundoff."""
    n = 10
    A = np.array([[1.0 / (i + j + 1) for j in range(n)] for i in range(n)], order="F")
    b = np.ones(n)
    Af = exact.to_frac_matrix(A.tolist())
    x_ex = exact.solve(Af, [Fraction(1)] * n)
    xm = max(abs(v) for v in x_ex)
    r = orc.gesv_dd(A, b, itermax=20)
    assert r["info"] == 0 and r["iter"] >= 2
    err = max(abs(a - e) for a, e in zip(_dd_frac(r["Xhi"], r["Xlo"]), x_ex))
    assert err <= 1e-16 * xm, float(err / xm)
    LU, piv, _ = orc.getrf(A)
    x0 = orc.getrs(LU, piv, b)
    err0 = max(abs(Fraction(float(a)) - e) for a, e in zip(x0, x_ex))
    assert err0 >= 1e-8 * xm  # the FP64 solve by itself is far less accurate


def test_gesv_dd_integer_system_exact(orc):
    """Integer A and integer x_true (b = A x_true exact in FP64): the
    double-double solution is x_true to within double-double rounding."""
    n = 40
    rng = np.random.default_rng(9)
    A = np.asfortranarray(rng.integers(-20, 21, (n, n)).astype(np.float64))
    A[np.diag_indices(n)] += 100.0
    xt = rng.integers(-1000, 1001, (n, 2)).astype(np.float64)
    B = A @ xt  # integers below 2^53: exact
    r = orc.gesv_dd(A, B)
    assert r["info"] == 0
    for c in range(2):
        for i in range(n):
            assert abs(Fraction(float(r["Xhi"][i, c])) + Fraction(float(r["Xlo"][i, c])) - int(xt[i, c])) \
                <= Fraction(1, 10 ** 20) * 1000


# ------------------------------------------- least squares (Section 6 extension)

def _ls_exact(A, b):
    """Exact rational least-squares solution from the normal equations."""
    Af = exact.to_frac_matrix(A.tolist())
    m, n = len(Af), len(Af[0])
    AtA = [[sum(Af[k][i] * Af[k][j] for k in range(m)) for j in range(n)] for i in range(n)]
    Atb = [sum(Af[k][i] * Fraction(float(b[k])) for k in range(m)) for i in range(n)]
    return exact.solve(AtA, Atb)


@pytest.mark.parametrize("m,n,seed", [(6, 3, 0), (8, 5, 1), (12, 4, 2), (5, 5, 3)])
def test_gels_aug_matches_exact_normal_equations(orc, m, n, seed):
    rng = np.random.default_rng(seed)
    A = rng.integers(-9, 10, (m, n)).astype(np.float64)
    b = rng.integers(-9, 10, m).astype(np.float64)
    x_ex = _ls_exact(A, b)
    if any(v.denominator == 0 for v in x_ex):
        pytest.skip("rank deficient")
    r = orc.gels_aug(A, b)
    assert r["info"] == 0
    x = r["X"][:, 0]
    sv = np.linalg.svd(A, compute_uv=False)
    k2 = sv[0] / sv[-1]
    xm = max(abs(float(v)) for v in x_ex)
    assert np.max(np.abs(x - np.array([float(v) for v in x_ex]))) <= 100 * k2 ** 2 * U64 * max(xm, 1.0)
    # the residual is orthogonal to the columns of A (normal equations)
    R = r["R"][:, 0]
    assert np.max(np.abs(A.T @ R)) <= 1e3 * U64 * np.max(np.abs(A)) * max(np.max(np.abs(R)), 1.0) * m
    assert np.allclose(R, b - A @ x, rtol=0, atol=1e-10 * max(np.max(np.abs(b)), 1.0))


def test_gels_aug_consistent_system(orc):
    """b in the range of A: the residual vanishes and x is the generating x."""
    rng = np.random.default_rng(5)
    A = rng.integers(-5, 6, (40, 10)).astype(np.float64)
    xt = rng.integers(-3, 4, 10).astype(np.float64)
    r = orc.gels_aug(A, A @ xt)
    assert np.max(np.abs(r["X"][:, 0] - xt)) <= 1e-12
    assert np.max(np.abs(r["R"])) <= 1e-11
