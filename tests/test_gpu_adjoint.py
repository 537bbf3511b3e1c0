"""GPU parity of the adjoint solve (reverse-mode derivative of X = A^{-1} B;
no counterpart in the paper): Bbar = A^{-T} G from the forward call's
low-precision factors with FP64 refinement against A^T, Abar = -Bbar X^T.

Checks, as for the forward solve: the transposed system's backward error
<= 1e-14 per column; Bbar and Abar against the closed form evaluated with the
oracle's FP64 solves (tolerance 10 kappa u64); central finite differences
(h = 1e-6) of L = sum(W * X) on 64 seeded entries of A and of B.
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


def _workspace(torch, mp, n, nrhs, prec, nb_outer=0, sym=False):
    import ctypes
    o = mp.default_opts(prec=prec, nb_outer=nb_outer)
    fn = mp.load().mp_posv_workspace_bytes if sym else mp.load().mp_gesv_workspace_bytes
    return mp.workspace(fn(n, nrhs, ctypes.byref(o)))


def _closed_form(orc, A, X, G):
    Bbar = orc.gesv_ir(np.asfortranarray(A.T), G, factor_prec=64)["X"].reshape(G.shape)
    return -Bbar @ X.T, Bbar


def _rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.mark.parametrize("prec,n,nrhs", [("fp16", 2048, 8), ("fp32", 300, 1), ("bf16", 777, 3),
                                         ("fp16x3", 1024, 2)])
def test_adjoint_closed_form(torch, mp, orc, prec, n, nrhs):
    A, B, Wt = inputs.adjoint_problem(n, nrhs, seed=n)
    dA = dev(torch, A)
    work = _workspace(torch, mp, n, nrhs, prec, nb_outer=128)
    X, _, st = mp.gesv(dA, dev(torch, B), prec=prec, nb_outer=128, work=work)
    assert st["flags"] == 0, st
    Abar, Bbar, sa = mp.gesv_adjoint(dA, X, dev(torch, Wt), work, prec=prec, nb_outer=128)
    assert sa["flags"] == 0 and sa["iter"] >= 0, sa
    Xh = host(X).reshape(n, nrhs)
    Bbar_h = host(Bbar).reshape(n, nrhs)
    bwd = orc.bwd_err(np.asfortranarray(A.T), Bbar_h, Wt)
    assert np.all(bwd <= 1e-14), bwd
    Abar_ref, Bbar_ref = _closed_form(orc, A, Xh, Wt)
    kappa = orc.kappa_inf(np.asfortranarray(A.T))
    assert _rel(Bbar_h, Bbar_ref) <= 10 * kappa * U64
    assert _rel(host(Abar), Abar_ref) <= 20 * kappa * U64


def test_adjoint_finite_differences(torch, mp, orc):
    n, nrhs = 128, 3
    A, B, Wt = inputs.adjoint_problem(n, nrhs, seed=11)
    work = _workspace(torch, mp, n, nrhs, "fp32")
    dA, dB = dev(torch, A), dev(torch, B)
    X, _, _ = mp.gesv(dA, dB, work=work)
    Abar, Bbar, _ = mp.gesv_adjoint(dA, X, dev(torch, Wt), work)
    Abar, Bbar = host(Abar), host(Bbar)

    def loss(Ap, Bp):
        Xp, _, st = mp.gesv(dev(torch, Ap), dev(torch, Bp))
        assert st["flags"] == 0
        return float(np.sum(Wt * host(Xp)))

    rng = np.random.default_rng(0)
    h = 1e-6
    for _ in range(64):
        i, j = rng.integers(0, n, 2)
        E = np.zeros_like(A)
        E[i, j] = h
        fd = (loss(A + E, B) - loss(A - E, B)) / (2 * h)
        assert abs(fd - Abar[i, j]) <= 1e-6 * np.max(np.abs(Abar)), (i, j, fd, Abar[i, j])
    for _ in range(64):
        i, c = rng.integers(0, n), rng.integers(0, nrhs)
        E = np.zeros_like(B)
        E[i, c] = h
        fd = (loss(A, B + E) - loss(A, B - E)) / (2 * h)
        assert abs(fd - Bbar[i, c]) <= 1e-6 * np.max(np.abs(Bbar)), (i, c, fd, Bbar[i, c])


def test_adjoint_after_cholesky(torch, mp, orc):
    n, nrhs = 500, 2
    A, B, _ = inputs.conditioned_system(n, 1e3, nrhs=nrhs, spd=True, seed=4)
    G = np.asfortranarray(np.random.default_rng(1).standard_normal((n, nrhs)))
    work = _workspace(torch, mp, n, nrhs, "fp32", sym=True)
    dA = dev(torch, A)
    X, st = mp.posv(dA, dev(torch, B), work=work)
    assert st["flags"] == 0
    Abar, Bbar, sa = mp.gesv_adjoint(dA, X, dev(torch, G), work)
    assert sa["flags"] == 0, sa
    Abar_ref, Bbar_ref = _closed_form(orc, A, host(X), G)
    kappa = orc.kappa_inf(A)
    assert _rel(host(Bbar), Bbar_ref) <= 10 * kappa * U64
    assert _rel(host(Abar), Abar_ref) <= 20 * kappa * U64


def test_adjoint_with_fp64_fallback_factors(torch, mp, orc):
    n = 8
    H = np.array([[1.0 / (i + j + 1) for j in range(n)] for i in range(n)], order="F")
    b = np.ones(n)
    g = np.linspace(-1.0, 1.0, n)
    work = _workspace(torch, mp, n, 1, "fp32")
    dH = dev(torch, H)
    X, _, st = mp.gesv(dH, dev(torch, b), work=work)
    assert st["flags"] & mp.FLAG_FALLBACK
    Abar, Bbar, sa = mp.gesv_adjoint(dH, X, dev(torch, g), work)
    assert sa["flags"] & mp.FLAG_FALLBACK and not sa["flags"] & mp.FLAG_NOT_CONVERGED, sa
    assert orc.bwd_err(np.asfortranarray(H.T), host(Bbar), g)[0] <= 1e-14


def test_solve_fn_autograd(torch, mp, orc):
    n, nrhs = 200, 2
    A, B, Wt = inputs.adjoint_problem(n, nrhs, seed=3)
    tA = dev(torch, A).requires_grad_(True)
    tB = dev(torch, B).requires_grad_(True)
    X = mp.solve_fn().apply(tA, tB)
    loss = (dev(torch, Wt) * X).sum()
    loss.backward()
    Abar_ref, Bbar_ref = _closed_form(orc, A, host(X), Wt)
    kappa = orc.kappa_inf(A)
    assert _rel(host(tB.grad), Bbar_ref) <= 10 * kappa * U64
    assert _rel(host(tA.grad), Abar_ref) <= 20 * kappa * U64


def test_adjoint_needs_forward_factors(torch, mp):
    n = 16
    work = _workspace(torch, mp, n, 1, "fp32")
    work.zero_()
    A = dev(torch, np.eye(n))
    with pytest.raises(mp.MpError):
        mp.gesv_adjoint(A, dev(torch, np.ones(n)), dev(torch, np.ones(n)), work)
