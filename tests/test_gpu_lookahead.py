"""The outer look-ahead of the blocked LU on the tensor-core rungs: after each
outer panel, the next panel's columns receive that panel's row moves, U12 and
trailing update first, the next panel is factored at once, and the same steps
for the columns further right (with the row moves over the columns to the
left) run concurrently on a second stream.  Checked through mp_getrf_lowp
and mp_gesv against the CPU oracle with the look-ahead forced on, at sizes
that span many outer panels and end in a ragged panel, and against the same
factorization with the look-ahead off.

Tolerances as for the plain blocked form (the same arithmetic per step):
pivots bit-exact on pivot-unambiguous matrices, ||PA - LU|| / ||A|| <= c n u_p,
|l_ij| <= 1, and solves with every column's bwd <= 1e-14 and the forward error
within 10 kappa_inf u64 of the oracle's FP64 solution.
"""
import numpy as np
import pytest

from paper_0808_2794_gb300 import inputs

pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53
U32 = 2.0 ** -24
UP = {"fp16x3": U32, "bf16": 2.0 ** -8, "fp16": 2.0 ** -11}


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
    return torch.from_numpy(np.asfortranarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def unambiguous_matrix(n, seed):
    """A = P0^T L0 U0 with |l_ij| <= 1/(2 sqrt(n)): exact partial pivoting
    picks the rows of P0 with a wide margin at every step, so no rounding
    order can change a pivot decision."""
    rng = np.random.default_rng(seed)
    L0 = np.tril(rng.uniform(-0.5, 0.5, (n, n)) / np.sqrt(n), -1) + np.eye(n)
    U0 = (np.triu(rng.uniform(-1, 1, (n, n)), 1) / np.sqrt(n)
          + np.diag(rng.uniform(1, 2, n) * rng.choice([-1, 1], n)))
    perm = rng.permutation(n)
    A = np.empty((n, n))
    A[perm, :] = L0 @ U0
    return np.asfortranarray(A)


def _factor(torch, mp, A, prec, nb, lookahead):
    W, _, _ = mp.convert(dev(torch, A))
    ipiv, info, flags = mp.getrf_lowp(W, prec=prec, nb_outer=nb, lookahead=lookahead)
    torch.cuda.synchronize()
    n = A.shape[0]
    return host(W)[:, :n].astype(np.float64), host(ipiv), info, flags


def _check_factors(A, LU, piv, u, c):
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


@pytest.mark.parametrize("n,nb", [(1000, 128), (2100, 256), (4133, 384)])
def test_lookahead_pivots_exact(torch, mp, orc, n, nb):
    """Every row exchange reaches every column: with unambiguous pivots the
    pivot sequence is the oracle's exactly and the factors satisfy the
    backward-error bound (a move missed or applied twice in any column range
    breaks the bound)."""
    A = unambiguous_matrix(n, seed=n)
    LU, piv, info, flags = _factor(torch, mp, A, "fp16x3", nb, 1)
    assert info == 0 and flags == 0
    _, pivo, _ = orc.getrf(A, prec=32)
    assert np.array_equal(piv, pivo)
    _check_factors(A, LU, piv, U32, c=8.0)


@pytest.mark.parametrize("prec", ["bf16", "fp16", "fp16x3"])
def test_lookahead_factor_bound(torch, mp, prec):
    """Random N(0,1) matrix over ten outer panels: the factors with the
    look-ahead on meet the same bound as with it off."""
    n = 2500
    A, _, _ = inputs.dense_system(n, seed=7)
    rel = []
    for la in (1, 0):
        LU, piv, info, flags = _factor(torch, mp, A, prec, 256, la)
        assert info == 0
        rel.append(_check_factors(A, LU, piv, UP[prec], c=4.0))
    assert rel[0] <= 4.0 * rel[1] + n * UP[prec], rel


@pytest.mark.parametrize("prec", ["fp16x3", "bf16"])
def test_lookahead_solve(torch, mp, orc, prec):
    """Whole solve, look-ahead on, n = 4096 + 37 (a ragged last panel) with
    two right-hand sides: FP64 accuracy, and the refinement needs about as
    many corrections as with the look-ahead off.  For bf16 the matrix gets a
    diagonal shift of 2 sqrt(n), so that kappa u_bf16 < 1 and the refinement
    converges without the FP64 fallback (Section 4)."""
    n = 4133
    A, B, _ = inputs.dense_system(n, nrhs=2, seed=11)
    if prec == "bf16":
        A = np.asfortranarray(A + 2.0 * np.sqrt(n) * np.eye(n))
    X1, _, st1 = mp.gesv(dev(torch, A), dev(torch, B), prec=prec, lookahead=1, refine="auto")
    X0, _, st0 = mp.gesv(dev(torch, A), dev(torch, B), prec=prec, lookahead=0, refine="auto")
    assert st1["iter"] >= 0 and not (st1["flags"] & 1), st1  # no FP64 fallback
    X1 = host(X1)
    bwd = orc.bwd_err(A, X1, B)
    assert np.all(bwd <= 1e-14), bwd
    ref = orc.gesv_ir(A, B, factor_prec=64)["X"].reshape(X1.shape)
    kappa = orc.kappa_inf(A)
    assert np.max(np.abs(X1 - ref)) / np.max(np.abs(ref)) <= 10 * kappa * U64
    assert abs(st1["iter"] - st0["iter"]) <= 2, (st1, st0)
