"""Pins of the CPU oracle for Algorithm 2 (Section 2.2), FGMRES(m_out) with
GMRES_SP(m_in) as its preconditioner, against what mathematics fixes
independently of the oracle's own code: exact rational minimal-residual
solutions over the Krylov space (GMRES's defining property), exact solves,
the degree of the minimal polynomial of a diagonal matrix, the flexible
Arnoldi relation, and exact integer products for the CSR product."""
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import exact, fgmres as fg
from paper_0808_2794_gb300 import inputs


def _csr(A):
    M = sp.csr_matrix(np.asarray(A, dtype=np.float64))
    M.sort_indices()
    return M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data.astype(np.float64)


def _int_matrix(n, seed, density=0.5, diag=20):
    rng = np.random.default_rng(seed)
    A = rng.integers(-9, 10, size=(n, n)) * (rng.random((n, n)) < density)
    A = A + np.diag(rng.integers(1, 9, size=n) + diag)
    return A.astype(np.float64)


@pytest.mark.parametrize("seed", range(3))
def test_csr_matvec_exact_on_integers(seed):
    """Integer matrix and vector: the CSR product equals the exact integer
    product (every partial sum is an integer below 2^53)."""
    A = _int_matrix(40, seed, density=0.2)
    x = np.random.default_rng(seed + 1).integers(-1000, 1000, size=40).astype(np.float64)
    ip, ix, d = _csr(A)
    y = fg.csr_matvec(ip, ix, d, x)
    want = [sum(int(A[i, j]) * int(x[j]) for j in range(40)) for i in range(40)]
    assert [int(v) for v in y] == want
    assert fg.norm_inf_csr(ip, d) == max(sum(abs(int(A[i, j])) for j in range(40)) for i in range(40))


def _krylov_minimiser(A, v, m):
    """Exact z* = K c* minimising ||v - A K c||_2 over the Krylov space
    K = [v, Av, ..., A^{m-1} v] (normal equations in rationals)."""
    n = len(v)
    Af = exact.to_frac_matrix(A.tolist())
    cols = [[Fraction(float(t)) for t in v]]
    for _ in range(m - 1):
        prev = cols[-1]
        cols.append([sum(Af[i][j] * prev[j] for j in range(n)) for i in range(n)])
    AK = [[sum(Af[i][l] * cols[c][l] for l in range(n)) for c in range(m)] for i in range(n)]
    vf = [Fraction(float(t)) for t in v]
    N = [[sum(AK[i][a] * AK[i][c] for i in range(n)) for c in range(m)] for a in range(m)]
    rhs = [sum(AK[i][a] * vf[i] for i in range(n)) for a in range(m)]
    c = exact.solve(N, rhs)
    return [float(sum(cols[k][i] * c[k] for k in range(m))) for i in range(n)]


@pytest.mark.parametrize("n,m,seed", [(6, 2, 0), (6, 3, 1), (8, 4, 2), (7, 5, 3)])
def test_gmres_cycle_is_the_krylov_minimal_residual_solution(n, m, seed):
    """GMRES's definition: after m steps from z = 0, z minimises ||v - A z||_2
    over the Krylov space of dimension m.  The FP64 cycle agrees with the exact
    rational minimiser found through the explicit Krylov basis."""
    A = _int_matrix(n, seed)
    v = np.random.default_rng(seed + 10).integers(-5, 6, size=n).astype(np.float64)
    v[0] = 7.0
    ip, ix, d = _csr(A)
    res = fg.arnoldi_cycle(lambda x: fg.csr_matvec(ip, ix, d, x), v, m, np.float64)
    assert res["steps"] == m
    want = np.array(_krylov_minimiser(A, v, m))
    assert np.max(np.abs(res["z"] - want)) <= 1e-11 * np.max(np.abs(want))
    # the last estimate is the true residual norm of z (in exact arithmetic)
    true_r = np.linalg.norm(v - A @ res["z"])
    assert abs(res["est"][-1] - true_r) <= 1e-10 * np.linalg.norm(v)


@pytest.mark.parametrize("seed", range(3))
def test_full_cycle_solves_exactly(seed):
    """m = n steps span the whole space: the cycle's z is A^{-1} v (against
    the exact rational solve)."""
    n = 8
    A = _int_matrix(n, seed, density=0.7, diag=3)
    v = np.arange(1.0, n + 1.0)
    ip, ix, d = _csr(A)
    res = fg.arnoldi_cycle(lambda x: fg.csr_matvec(ip, ix, d, x), v, n, np.float64)
    want = [float(t) for t in exact.solve(exact.to_frac_matrix(A.tolist()), [Fraction(t) for t in v])]
    assert np.max(np.abs(res["z"] - np.array(want))) <= 1e-10 * max(abs(t) for t in want)


def test_diagonal_matrix_minimal_polynomial_degree():
    """A diagonal matrix with d distinct eigenvalues: the Krylov space of
    dimension d contains A^{-1} v, so GMRES ends exactly at step d (breakdown
    or zero estimate), with a non-zero estimate at step d - 1."""
    vals = np.array([1.0, 2.0, 2.0, 5.0, 5.0, 5.0, -3.0, 7.0, 7.0])
    d = len(set(vals.tolist()))
    A = np.diag(vals)
    v = np.ones(len(vals))
    ip, ix, dd = _csr(A)
    res = fg.arnoldi_cycle(lambda x: fg.csr_matvec(ip, ix, dd, x), v, len(vals), np.float64,
                           stop_rel=1e-13)
    assert res["steps"] == d
    assert res["est"][d - 2] > 1e-3
    assert np.max(np.abs(res["z"] - v / vals)) <= 1e-12


def test_identity_one_step():
    n = 10
    ip, ix, d = _csr(np.eye(n))
    v = np.linspace(-1, 1, n)
    res = fg.arnoldi_cycle(lambda x: fg.csr_matvec(ip, ix, d, x), v, 5, np.float64, stop_rel=1e-14)
    assert res["steps"] == 1 and np.max(np.abs(res["z"] - v)) <= 1e-15


def test_flexible_arnoldi_relation():
    """FGMRES's Arnoldi relation with a varying preconditioner:
    A Z_k = V_{k+1} H_k and V orthonormal, to FP64 rounding."""
    n, m = 60, 8
    ip, ix, d, _, _, _ = inputs.sparse_system("cage11_like", scale=60 / 39082)
    n = len(ip) - 1
    rng = np.random.default_rng(3)
    calls = []

    def precond(v):  # a different (nonlinear) preconditioner at every step
        calls.append(1)
        return v * (1.0 + 0.1 * len(calls)) + 0.01 * rng.standard_normal(n)

    r0 = rng.standard_normal(n)
    res = fg.arnoldi_cycle(lambda x: fg.csr_matvec(ip, ix, d, x), r0, m, np.float64, precond=precond)
    k = res["steps"]
    V = np.array(res["V"][: k + 1]).T
    Z = np.array(res["Z"][:k]).T
    A = sp.csr_matrix((d, ix, ip), shape=(n, n))
    lhs = A @ Z
    rhs = V @ res["H"]
    assert np.max(np.abs(lhs - rhs)) <= 1e-12 * np.max(np.abs(lhs))
    # modified Gram-Schmidt keeps orthogonality to O(u) times the basis condition
    assert np.max(np.abs(V.T @ V - np.eye(k + 1))) <= 1e-10


def test_fgmres_with_exact_inner_solve_converges_in_one_step():
    """If the inner solve returns A^{-1} v exactly, the first outer step's
    z_1 = A^{-1} r / beta already solves the system: one cycle, one step."""
    ip, ix, d, b, xt, _ = inputs.sparse_system("cage11_like", scale=200 / 39082, seed=2)
    n = len(ip) - 1
    A = sp.csr_matrix((d, ix, ip), shape=(n, n)).toarray()
    res = fg.fgmres(ip, ix, d, b, m_out=5, m_in=0, inner_solve=lambda v: np.linalg.solve(A, v))
    assert res["converged"] and res["cycles"] == 1 and res["outer_steps"] == 1


@pytest.mark.parametrize("name", ["cage11_like", "poisson3db_like", "sio_like"])
def test_fgmres_sp_reaches_fp64_accuracy(name):
    """Algorithm 2 with the inner GMRES in FP32 on small stand-ins of the
    Table 2 matrices: the backward error reaches 1e-14 and the forward error
    is within 10 kappa_inf u64 of the exact solution (dense inverse for kappa)."""
    scale = {"cage11_like": 600 / 39082, "poisson3db_like": 9 / 44, "sio_like": 600 / 33401}[name]
    ip, ix, d, b, xt, cfg = inputs.sparse_system(name, scale=scale, seed=1)
    n = len(ip) - 1
    res = fg.fgmres(ip, ix, d, b, cfg["m_out"], cfg["m_in"], inner=np.float32)
    assert res["converged"] and res["bwd"] <= 1e-14, res["hist"]
    A = sp.csr_matrix((d, ix, ip), shape=(n, n)).toarray()
    x = np.linalg.solve(A, b)
    kappa = np.linalg.norm(A, np.inf) * np.linalg.norm(np.linalg.inv(A), np.inf)
    fwd = np.max(np.abs(res["x"] - x)) / np.max(np.abs(x))
    assert fwd <= 10 * kappa * 2.0 ** -53 + 1e-15, (fwd, kappa)
    # the FP32 inner solves are exercised: more than one inner step per outer step
    assert res["inner_steps"] > res["outer_steps"]


def test_restarted_gmres_and_dp_inner_agree():
    """The comparison methods: plain restarted GMRES(m) in FP64 and
    FGMRES-GMRES_DP reach the same solution as FGMRES-GMRES_SP."""
    ip, ix, d, b, xt, cfg = inputs.sparse_system("poisson3db_like", scale=8 / 44, seed=4)
    r_sp = fg.fgmres(ip, ix, d, b, cfg["m_out"], cfg["m_in"], inner=np.float32)
    r_dp = fg.fgmres(ip, ix, d, b, cfg["m_out"], cfg["m_in"], inner=np.float64)
    r_g = fg.gmres_restarted(ip, ix, d, b, cfg["m"])
    assert r_sp["converged"] and r_dp["converged"] and r_g["converged"]
    scale = np.max(np.abs(r_sp["x"]))
    assert np.max(np.abs(r_sp["x"] - r_dp["x"])) <= 1e-11 * scale
    assert np.max(np.abs(r_sp["x"] - r_g["x"])) <= 1e-11 * scale


def test_fp32_inner_cycle_rounds_the_matrix():
    """GMRES_SP works on the FP32-rounded matrix: with an FP64 inner cycle of
    full dimension the preconditioned step is exact, with the FP32 one its
    accuracy is limited to about u32 (so the outer loop has work to do)."""
    ip, ix, d, b, xt, _ = inputs.sparse_system("cage11_like", scale=40 / 39082, seed=5)
    n = len(ip) - 1
    A = sp.csr_matrix((d, ix, ip), shape=(n, n)).toarray()
    v = b / np.linalg.norm(b)
    z64 = fg.gmres_cycle(ip, ix, d, v, n, np.float64)["z"]
    z32 = fg.gmres_cycle(ip, ix, d, v, n, np.float32)["z"].astype(np.float64)
    zt = np.linalg.solve(A, v)
    e64 = np.max(np.abs(z64 - zt)) / np.max(np.abs(zt))
    e32 = np.max(np.abs(z32 - zt)) / np.max(np.abs(zt))
    assert e64 <= 1e-12 and 1e-9 <= e32 <= 1e-4
