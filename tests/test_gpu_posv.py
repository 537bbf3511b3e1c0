"""GPU parity of the Cholesky variant (Section 3.1.1: SPOTRF, SPOTRS and the
symmetric residual take the places of SGETRF, SGETRS and DGEMM in
Algorithm 1; Section 6), through the C ABI, against the CPU oracle.

Tolerances: the factor satisfies ||A - L L^T||_inf / ||A||_inf <= c n u_p
(the oracle's own FP32 factor is held to the same bound); a solve must give
every column bwd <= 1e-14 and ||x - x_oracle|| / ||x_oracle|| <= 10
kappa_inf(A) 2^-53, with x_oracle from the oracle's FP64 solve.
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


def _potrf(torch, mp, A, prec="fp32", nb_outer=0):
    n = A.shape[0]
    ld = mp.factor_ld(n)
    W = torch.zeros((n, ld), dtype=torch.float32, device="cuda")
    W[:, :n] = torch.from_numpy(np.tril(A).astype(np.float32)).cuda()  # row-major: W[i, j] = a_ij
    info, flags = mp.potrf_lowp(W, prec=prec, nb_outer=nb_outer)
    return np.tril(host(W)[:, :n].astype(np.float64)), info, flags


@pytest.mark.parametrize("n,nb", [(1, 0), (31, 0), (33, 32), (100, 64), (513, 128), (1500, 256)])
def test_potrf_fp32_backward_bound(torch, mp, orc, n, nb):
    A, _, _ = inputs.conditioned_system(n, 1e3, spd=True, seed=n)
    L, info, flags = _potrf(torch, mp, A, nb_outer=nb)
    assert info == 0 and flags == 0
    assert np.all(np.diag(L) > 0)
    An = np.max(np.sum(np.abs(A), axis=1))
    res = np.max(np.sum(np.abs(A - L @ L.T), axis=1)) / An
    Lo, info_o = orc.potrf(A, prec=32)
    Lo = np.tril(Lo)
    res_o = np.max(np.sum(np.abs(A - Lo @ Lo.T), axis=1)) / An
    assert info_o == 0
    assert res <= 4 * n * U32 and res_o <= 4 * n * U32, (res, res_o)


@pytest.mark.parametrize("prec", ["bf16", "fp16", "fp16x3"])
def test_potrf_lowp_backward_bound(torch, mp, orc, prec):
    n = 1500
    A, _, _ = inputs.conditioned_system(n, 1e2, spd=True, seed=3)
    L, info, flags = _potrf(torch, mp, A, prec=prec, nb_outer=256)
    assert info == 0
    An = np.max(np.sum(np.abs(A), axis=1))
    res = np.max(np.sum(np.abs(A - L @ L.T), axis=1)) / An
    assert res <= 4 * n * UP[prec], res


def test_potrf_reports_leading_minor(torch, mp):
    n = 70
    A = np.eye(n)
    A[40, 40] = -1.0
    _, info, flags = _potrf(torch, mp, A)
    assert info == 41 and flags & mp.FLAG_LOWP_BREAKDOWN


@pytest.mark.parametrize("n,nrhs", [(1, 1), (2, 1), (31, 2), (64, 1), (129, 3), (700, 1), (2048, 4)])
def test_posv_fp32(torch, mp, orc, n, nrhs):
    A, B, _ = inputs.conditioned_system(n, 1e4, nrhs=nrhs, spd=True, seed=n + 1)
    X, st = mp.posv(dev(torch, A), dev(torch, B))
    X = host(X).reshape(n, nrhs)
    assert st["flags"] == 0 and st["iter"] >= 0, st
    _check_solution(orc, A, B, X)
    r = orc.posv_ir(A, B, factor_prec=32)
    assert st["iter"] <= 2 * r["iter"] + 3, (st["iter"], r["iter"])


def test_posv_reads_lower_triangle_only(torch, mp, orc):
    n = 300
    A, B, _ = inputs.conditioned_system(n, 1e3, nrhs=2, spd=True, seed=5)
    An = A.copy(order="F")
    An[np.triu_indices(n, 1)] = np.nan
    X, st = mp.posv(dev(torch, An), dev(torch, B))
    assert st["flags"] == 0, st
    _check_solution(orc, A, B, host(X))


@pytest.mark.parametrize("prec,kappa", [("bf16", 10.0), ("fp16", 1e2), ("fp16x3", 1e5)])
@pytest.mark.parametrize("n", [300, 1100, 2048])
def test_posv_lowp(torch, mp, orc, prec, kappa, n):
    A, B, _ = inputs.conditioned_system(n, kappa, spd=True, seed=n + 2)
    X, st = mp.posv(dev(torch, A), dev(torch, B), prec=prec, nb_outer=128)
    assert not st["flags"] & mp.FLAG_FALLBACK, st
    _check_solution(orc, A, B, host(X).reshape(n, 1))


def test_posv_gmres_beyond_classical(torch, mp, orc):
    """kappa u_16 >> 1: classical refinement with FP16 Cholesky factors
    cannot contract; GMRES with the same factors converges (Section 4)."""
    n = 1024
    A, B, _ = inputs.conditioned_system(n, 1e5, spd=True, seed=8)
    dA, dB = dev(torch, A), dev(torch, B)
    X, st = mp.posv(dA, dB, prec="fp16", nb_outer=128, allow_fallback=False)
    assert st["flags"] & (mp.FLAG_STALLED | mp.FLAG_NOT_CONVERGED | mp.FLAG_LOWP_BREAKDOWN), st
    X, st = mp.posv(dA, dB, prec="fp16", nb_outer=128, refine="gmres", allow_fallback=False)
    assert st["flags"] == mp.FLAG_GMRES_USED, st
    _check_solution(orc, A, B, host(X).reshape(n, 1))


def test_posv_not_positive_definite(torch, mp):
    n = 50
    A = np.asfortranarray(np.diag(np.linspace(1.0, 2.0, n)))
    A[9, 9] = -3.0
    X, st = mp.posv(dev(torch, A), dev(torch, np.ones(n)))
    assert st["info_fp64"] == 10 and st["flags"] & mp.FLAG_FALLBACK, st
    assert st["info"] == 10


def test_posv_ill_conditioned_falls_back(torch, mp, orc):
    n = 9
    H = np.array([[1.0 / (i + j + 1) for j in range(n)] for i in range(n)], order="F")
    b = np.ones(n)
    X, st = mp.posv(dev(torch, H), dev(torch, b))
    assert st["flags"] & mp.FLAG_FALLBACK and st["iter"] == -1, st
    assert orc.bwd_err(H, host(X), b)[0] <= 1e-14


def test_posv_argument_errors(torch, mp):
    A = dev(torch, np.eye(4))
    with pytest.raises(mp.MpError):
        mp.posv(A, dev(torch, np.ones(4)), itermax=-1)
