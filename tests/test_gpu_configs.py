"""GPU parity at the configurations the solver is specified for, beyond the
dense headline: general systems of prescribed condition number (the paper's
Section 4 / Fig. 4 protocol at n = 4096, nrhs = 4, FP16 factors, classical
refinement against GMRES-based refinement), the plain FP64 solve (prec=fp64,
the comparator of the paper's Table 3 speedups), and the adjoint at n = 2048,
nrhs = 8 against central finite differences.

Tolerances are those of every whole-solve test: per-column backward error
<= 1e-14 from the oracle's compensated residual, forward error within
20 kappa_inf(A) 2^-53 of X_true where kappa_inf comes from the closed-form
inverse, or within 10 kappa_inf 2^-53 of the oracle's FP64 solution.
"""
import numpy as np
import pytest

from paper_0808_2794_gb300 import inputs

pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53
KAPPAS = (1e2, 1e4, 1e6, 1e8)


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


@pytest.fixture(scope="module")
def general_family():
    """A = U diag(s) V^T for every kappa (Haar U, V drawn once; the same arrays
    as conditioned_system(4096, kappa, nrhs=4, seed=0)), with kappa_inf(A) from
    the closed-form inverse V diag(1/s) U^T."""
    n = 4096
    rng = np.random.default_rng(0)
    U = inputs.haar_orthogonal(rng, n)
    V = inputs.haar_orthogonal(rng, n)
    out = {}
    for kappa, A, B, X in inputs.conditioned_family(n, KAPPAS, nrhs=4, spd=False, seed=0):
        s = kappa ** (-np.arange(n, dtype=np.float64) / (n - 1))
        Ainv = (V / s[None, :]) @ U.T
        kinf = np.max(np.sum(np.abs(A), axis=1)) * np.max(np.sum(np.abs(Ainv), axis=1))
        out[kappa] = (A, B, X, kinf)
    return out


@pytest.mark.parametrize("refine", ["classical", "gmres"])
@pytest.mark.parametrize("kappa", KAPPAS)
def test_general_lu_n4096_fp16_prescribed_kappa(torch, mp, orc, general_family, kappa, refine):
    """FP16 LU of A = U diag(s) V^T: every column reaches bwd <= 1e-14 and the
    forward error is within 20 kappa_inf u64 of X_true, whichever of
    classical refinement, GMRES refinement or the FP64 fallback answers.
    kappa * u16 < 1 (kappa = 1e2): classical refinement converges on its own;
    GMRES refinement, preconditioned by the same factors, also converges at
    kappa = 1e4 where classical refinement cannot (Section 4)."""
    A, B, X_true, kinf = general_family[kappa]
    X, piv, st = mp.gesv(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), prec="fp16", refine=refine)
    X = X.cpu().numpy()
    assert np.all(orc.bwd_err(A, X, B) <= 1e-14), st
    fwd = np.max(np.abs(X - X_true)) / np.max(np.abs(X_true))
    assert fwd <= 20 * kinf * U64, (fwd, kinf, st)
    if kappa <= 1e2:
        assert st["flags"] & mp.FLAG_FALLBACK == 0, st
    if refine == "gmres" and kappa <= 1e4:
        assert st["flags"] & mp.FLAG_FALLBACK == 0 and st["flags"] & mp.FLAG_GMRES_USED, st


@pytest.mark.parametrize("n,nrhs,seed", [(1, 1, 0), (37, 2, 1), (1000, 3, 2), (4096, 1, 3)])
def test_plain_fp64_solve(torch, mp, orc, n, nrhs, seed):
    """prec=fp64: FP64 LU with partial pivoting and FP64 solves on the GPU, no
    low precision.  The pivots are those of the oracle's FP64 LU wherever the
    pivot choice is unambiguous (checked up to the first near tie), the
    solution is within 10 kappa_inf u64 of the oracle's FP64 solution and the
    FALLBACK flag is never set."""
    A, B, _ = inputs.dense_system(n, nrhs=nrhs, seed=seed)
    X, piv, st = mp.gesv(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), prec="fp64")
    assert st["flags"] & (mp.FLAG_FALLBACK | mp.FLAG_LOWP_BREAKDOWN) == 0, st
    assert st["iter"] >= 0
    X = X.cpu().numpy().reshape(n, nrhs)
    assert np.all(orc.bwd_err(A, X, B) <= 1e-14)
    LU, piv_or, info = orc.getrf(A)
    x_or = orc.gesv_ir(A, B, factor_prec=64)["X"].reshape(n, nrhs)
    kinf = orc.kappa_inf_est_lu(A, LU, piv_or) if n > 1000 else orc.kappa_inf(A)
    assert np.max(np.abs(X - x_or)) / np.max(np.abs(x_or)) <= 10 * kinf * U64
    p = piv.cpu().numpy()
    if n <= 1000:
        # pivots agree up to the first step where two candidates are within
        # a relative 1e-12 (the two sides round the updates differently)
        first_diff = np.argmax(p != piv_or) if np.any(p != piv_or) else n
        assert first_diff == n or _near_tie(A, piv_or, first_diff), (first_diff, p[:first_diff + 1])


def _near_tie(A, piv, k):
    """True if, at elimination step k of the FP64 GEPP with pivots piv, the
    two largest candidate magnitudes are within a relative 1e-12."""
    M = np.array(A, dtype=np.float64, order="F", copy=True)
    for j in range(k):
        p = piv[j] - 1
        if p != j:
            M[[j, p], :] = M[[p, j], :]
        M[j + 1:, j] /= M[j, j]
        M[j + 1:, j + 1:] -= np.outer(M[j + 1:, j], M[j, j + 1:])
    mags = np.sort(np.abs(M[k:, k]))[::-1]
    return len(mags) > 1 and mags[0] - mags[1] <= 1e-12 * mags[0]


def test_plain_fp64_cholesky(torch, mp, orc):
    A, B, X_true = inputs.conditioned_system(700, 1e6, nrhs=2, spd=True, seed=5)
    X, st = mp.posv(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), prec="fp64")
    assert st["flags"] & (mp.FLAG_FALLBACK | mp.FLAG_LOWP_BREAKDOWN) == 0, st
    X = X.cpu().numpy()
    assert np.all(orc.bwd_err(A, X, B) <= 1e-14)
    x_or = orc.posv_ir(A, B, factor_prec=64)["X"]
    assert np.max(np.abs(X - x_or)) / np.max(np.abs(x_or)) <= 10 * orc.kappa_inf(A) * U64


def test_plain_fp64_singular_reports_info(torch, mp, orc):
    """A zero column keeps its pivot exactly zero at every step: LAPACK's
    info = its 1-based index, as the oracle's FP64 LU reports."""
    n = 64
    A = inputs.small_integer_matrix(n, seed=9)
    A[:, 17] = 0.0
    assert orc.getrf(A)[2] == 18
    _, _, st = mp.gesv(torch.from_numpy(A).cuda(), torch.from_numpy(np.ones(n)).cuda(), prec="fp64")
    assert st["info_fp64"] == 18, st


def test_adjoint_finite_differences_n2048(torch, mp):
    """The adjoint workload's own size: n = 2048, nrhs = 8, A = N(0,1) + sqrt(n) I,
    FP16 factors refined to FP64; loss = sum(W * X).  Central differences
    (h = 1e-6) of the loss on 64 seeded entries of A and 64 of B agree with
    Abar and Bbar to 1e-6 of their largest magnitude (truncation O(h^2) plus
    rounding O(u/h) in the loss)."""
    import ctypes
    n, nrhs = 2048, 8
    A, B, Wt = inputs.adjoint_problem(n, nrhs, seed=0)
    o = mp.default_opts(prec="fp16")
    lib = mp.load()
    work = mp.workspace(lib.mp_gesv_workspace_bytes(n, nrhs, ctypes.byref(o)))
    dA, dB, dW = (torch.from_numpy(x).cuda() for x in (A, B, Wt))
    X, _, st = mp.gesv(dA, dB, prec="fp16", work=work)
    assert st["flags"] == 0, st
    Abar, Bbar, sa = mp.gesv_adjoint(dA, X, dW, work, prec="fp16")
    assert sa["flags"] == 0, sa
    Abar, Bbar = Abar.cpu().numpy(), Bbar.cpu().numpy()
    fwork = mp.workspace(lib.mp_gesv_workspace_bytes(n, nrhs, ctypes.byref(o)))

    def loss(Ap, Bp):
        Xp, _, s2 = mp.gesv(Ap, Bp, prec="fp16", work=fwork)
        assert s2["flags"] == 0, s2
        return float((dW * Xp).sum())

    rng = np.random.default_rng(0)
    h = 1e-6
    amax, bmax = np.max(np.abs(Abar)), np.max(np.abs(Bbar))
    for _ in range(64):
        i, j = (int(v) for v in rng.integers(0, n, 2))
        Ap, Am = dA.clone(), dA.clone()
        Ap[i, j] += h
        Am[i, j] -= h
        fd = (loss(Ap, dB) - loss(Am, dB)) / (2 * h)
        assert abs(fd - Abar[i, j]) <= 1e-6 * amax, (i, j, fd, Abar[i, j])
    for _ in range(64):
        i, c = int(rng.integers(0, n)), int(rng.integers(0, nrhs))
        Bp, Bm = dB.clone(), dB.clone()
        Bp[i, c] += h
        Bm[i, c] -= h
        fd = (loss(dA, Bp) - loss(dA, Bm)) / (2 * h)
        assert abs(fd - Bbar[i, c]) <= 1e-6 * bmax, (i, c, fd, Bbar[i, c])
