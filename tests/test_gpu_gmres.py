"""GPU parity of GMRES-based refinement (Section 2.2: right-preconditioned
Krylov solve of A d = r with M = (LU)^{-1} P from the low-precision factors;
Section 4: its convergence reaches further in kappa than classical
refinement).

Tolerances are those of the whole-solve tests: every column bwd <= 1e-14 and
||x - x_oracle|| / ||x_oracle|| <= 10 kappa_inf(A) 2^-53.  Iteration counts
are compared with the oracle's GMRES refinement (FP32 factors) only as a
sanity bound: the two sides orthogonalise and round differently.
"""
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


def dev(torch, a):
    a = np.asarray(a)
    if a.ndim == 1:
        return torch.from_numpy(a.copy()).cuda()
    return torch.from_numpy(np.asfortranarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def _check_solution(orc, A, B, X):
    bwd = orc.bwd_err(A, X, B)
    assert np.all(bwd <= 1e-14), bwd
    ref = orc.gesv_ir(A, B, factor_prec=64)["X"].reshape(X.shape)
    kappa = orc.kappa_inf(A)
    fwd = np.max(np.abs(X - ref)) / np.max(np.abs(ref))
    assert fwd <= 10 * kappa * U64, (fwd, kappa)


@pytest.mark.parametrize("n,nrhs", [(1, 1), (5, 1), (64, 2), (300, 1), (1024, 3)])
def test_gmres_fp32_dense(torch, mp, orc, n, nrhs):
    A, B, _ = inputs.dense_system(n, nrhs=nrhs, seed=n + 11)
    X, piv, st = mp.gesv(dev(torch, A), dev(torch, B), prec="fp32", refine="gmres")
    X = host(X).reshape(n, nrhs)
    assert st["flags"] == mp.FLAG_GMRES_USED, st
    _check_solution(orc, A, B, X)
    # the oracle's GMRES refinement (FP32 LU, MGS) on the first column;
    # the device loop adds one outer step to confirm the FP64 floor
    r = orc.gmres_ir(A, B[:, 0])
    assert r["bwd"] <= 1e-14
    assert 0 <= st["iter"] <= r["outer"] + 2, (st["iter"], r)


@pytest.mark.parametrize("prec,kappa", [("fp16", 1e4), ("bf16", 1e3)])
def test_gmres_converges_where_classical_stalls(torch, mp, orc, prec, kappa):
    """kappa u_p > 1: the classical loop cannot contract (Section 4), the
    preconditioned Krylov solve still reaches FP64 accuracy without falling
    back to the FP64 factorization."""
    n = 1024
    A, B, _ = inputs.conditioned_system(n, kappa, seed=1)
    dA, dB = dev(torch, A), dev(torch, B)
    X, _, st = mp.gesv(dA, dB, prec=prec, nb_outer=128, allow_fallback=False)
    assert st["flags"] & (mp.FLAG_STALLED | mp.FLAG_NOT_CONVERGED), st
    X, _, st = mp.gesv(dA, dB, prec=prec, nb_outer=128, refine="gmres", allow_fallback=False)
    assert st["flags"] == mp.FLAG_GMRES_USED, st
    _check_solution(orc, A, B, host(X).reshape(n, 1))
    X, _, st = mp.gesv(dA, dB, prec=prec, nb_outer=128, refine="auto")
    assert st["flags"] & mp.FLAG_GMRES_USED and not st["flags"] & mp.FLAG_FALLBACK, st
    _check_solution(orc, A, B, host(X).reshape(n, 1))


def test_gmres_auto_keeps_classical_when_it_converges(torch, mp, orc):
    A, B, _ = inputs.dense_system(500, nrhs=2, seed=3)
    X, _, st = mp.gesv(dev(torch, A), dev(torch, B), prec="fp32", refine="auto")
    assert st["flags"] == 0, st
    _check_solution(orc, A, B, host(X))


def test_gmres_hopeless_falls_back(torch, mp, orc):
    """kappa u_p far above 1: GMRES(30) cannot make progress either; the
    answer comes from the FP64 factorization."""
    n = 512
    A, B, _ = inputs.conditioned_system(n, 1e7, seed=2)
    X, _, st = mp.gesv(dev(torch, A), dev(torch, B), prec="bf16", nb_outer=128, refine="gmres",
                       itermax=6)
    assert st["flags"] & mp.FLAG_FALLBACK and st["iter"] == -1, st
    assert np.all(orc.bwd_err(A, host(X).reshape(n, 1), B) <= 1e-14)


def test_gmres_restart_and_tol_arguments(torch, mp, orc):
    A, B, _ = inputs.dense_system(200, seed=4)
    dA, dB = dev(torch, A), dev(torch, B)
    for m in (1, 2, 64):
        X, _, st = mp.gesv(dA, dB, refine="gmres", gmres_restart=m)
        assert st["flags"] == mp.FLAG_GMRES_USED, (m, st)
        _check_solution(orc, A, B, host(X).reshape(200, 1))
    with pytest.raises(mp.MpError):
        mp.gesv(dA, dB, refine="gmres", gmres_restart=0)
    with pytest.raises(mp.MpError):
        mp.gesv(dA, dB, refine="gmres", gmres_tol=1.0)
