"""Parity at the full sizes of the measured workloads, in the configuration
the benchmark times (default options: the fp16x3 rung, classical
refinement).  The oracle checks what it can afford at these sizes: the
backward error of every column from its compensated (Dot2) FP64 residual over
the whole matrix, and, where the condition number is known in closed form,
the forward error.
"""
import os

import numpy as np
import pytest

from paper_0808_2794_gb300 import inputs

pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53


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


def test_dense_lu_n16384_bench_configuration(torch, mp, orc):
    """The benchmark's workload: n = 16384, A ~ N(0,1), x ~ U[-1,1], b = A x."""
    n = 16384
    A, B, X_true = inputs.dense_system(n, seed=0)
    X, piv, st = mp.gesv(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda())
    assert st["flags"] == 0 and st["iter"] >= 1, st
    X = X.cpu().numpy().reshape(n, 1)
    assert np.all(orc.bwd_err(A, X, B) <= 1e-14)
    p = piv.cpu().numpy()
    assert np.all((p >= np.arange(1, n + 1)) & (p <= n))  # LAPACK ipiv: row k swapped with ipiv[k] >= k
    # the solution agrees with x_true to well inside the FP32-factor regime
    assert np.max(np.abs(X[:, 0] - X_true[:, 0])) / np.max(np.abs(X_true)) <= 1e-9


@pytest.mark.slow
def test_dense_lu_n16384_against_oracle_fp64(torch, mp, orc):
    """The benchmark's workload and launch configuration, against the
    oracle's FP64 solve of the same system: one FP64 LU with partial pivoting
    on the host cores (about 1.5 minutes on 16 cores), x_or from it with one
    FP64 correction from the compensated residual, and kappa_inf(A) estimated
    from the same factors (Hager-Higham, a lower bound).  The GPU solution is
    within 10 kappa_inf u64 of x_or and every column's backward error, from
    the oracle's compensated residual, is <= 1e-14."""
    n = 16384
    A, B, X_true = inputs.dense_system(n, seed=0)
    X, piv, st = mp.gesv(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), prec="fp16x3")
    assert st["flags"] == 0, st
    X = X.cpu().numpy().reshape(n, 1)
    assert np.all(orc.bwd_err(A, X, B) <= 1e-14)
    orc.set_threads(os.cpu_count() or 1)
    LU, piv_or, info = orc.getrf(A)
    assert info == 0
    x0 = orc.getrs(LU, piv_or, B).reshape(n, 1)
    r = orc.residual(A, x0, B, compensated=True).reshape(n, 1)
    x_or = x0 + orc.getrs(LU, piv_or, r).reshape(n, 1)
    kinf = orc.kappa_inf_est_lu(A, LU, piv_or)
    fwd = np.max(np.abs(X - x_or)) / np.max(np.abs(x_or))
    assert fwd <= 10 * kinf * U64, (fwd, kinf)


@pytest.mark.parametrize("n", [20480, 33024])
def test_dense_lu_tall_panel_variants(torch, mp, orc, n):
    """Sizes whose first leaves are taller than 16384 rows (16-column leaves,
    4 rows per thread) and, at n = 33024, taller than 32768 rows (8-column
    leaves, 8 rows per thread), so the panel kernel's taller variants run the
    whole leaf pipeline.  Too large for an oracle solve: the backward error
    comes from the oracle's compensated residual over the whole matrix (an
    O(n^2) pass), the forward error from the known x_true."""
    A, B, X_true = inputs.dense_system(n, seed=3)
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    X, piv, st = mp.gesv(Ad, Bd)
    assert st["flags"] == 0, st
    del Ad
    X = X.cpu().numpy().reshape(n, 1)
    orc.set_threads(os.cpu_count() or 1)
    bwd = orc.bwd_err(A, X, B)
    assert np.all(bwd <= 1e-14), (bwd, st)
    assert np.max(np.abs(X[:, 0] - X_true[:, 0])) / np.max(np.abs(X_true)) <= 1e-8


@pytest.mark.parametrize("kappa", [1e2, 1e4, 1e6, 1e8])
def test_spd_n4096_fp16_prescribed_kappa(torch, mp, orc, kappa):
    """SPD systems of prescribed condition number (the paper's Fig. 4
    protocol), n = 4096, nrhs = 4, FP16 Cholesky with automatic GMRES
    continuation and FP64 fallback: every column reaches bwd <= 1e-14 and the
    forward error is within 20 kappa_inf u64 of X_true (kappa_inf from the
    closed-form inverse U diag(1/s) U^T)."""
    n, nrhs = 4096, 4
    A, B, X_true = inputs.conditioned_system(n, kappa, nrhs=nrhs, spd=True, seed=0)
    X, st = mp.posv(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), prec="fp16", refine="auto")
    X = X.cpu().numpy()
    assert np.all(orc.bwd_err(A, X, B) <= 1e-14), st
    # closed-form inverse: A = U diag(s) U^T with the generator's U and s
    rng = np.random.default_rng(0)
    U = inputs.haar_orthogonal(rng, n)
    s = kappa ** (-np.arange(n, dtype=np.float64) / (n - 1))
    Ainv = (U / s[None, :]) @ U.T
    kinf = np.max(np.sum(np.abs(A), axis=1)) * np.max(np.sum(np.abs(Ainv), axis=1))
    fwd = np.max(np.abs(X - X_true)) / np.max(np.abs(X_true))
    assert fwd <= 20 * kinf * U64, (fwd, kinf, st)
    if kappa <= 1e4:
        assert not st["flags"] & mp.FLAG_FALLBACK, st
