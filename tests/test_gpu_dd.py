"""GPU parity of refinement with an extra-precise residual (Section 5,
QDGESV; double-double in place of quadruple precision): FP64 factors, the
residual b - A (xhi + xlo) accumulated in double-double, the solution kept in
double-double.  Compared with the oracle's restatement of the same algorithm
and with exact rational solutions: both reach the double-double level
kappa u_dd, far below FP64's kappa u64.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import exact
from paper_0808_2794_gb300 import inputs

pytestmark = pytest.mark.gpu

UDD = 2.0 ** -104


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


def _uniform(n, nrhs, seed):
    """The paper's Section 5 matrices: entries uniform in (-1, 1)."""
    rng = np.random.default_rng(seed)
    A = np.asfortranarray(rng.uniform(-1.0, 1.0, (n, n)))
    B = np.asfortranarray(rng.uniform(-1.0, 1.0, (n, nrhs)))
    return A, B


@pytest.mark.parametrize("n,nrhs", [(1, 1), (100, 1), (513, 2), (1000, 1)])
def test_dd_matches_oracle(torch, mp, orc, n, nrhs):
    A, B = _uniform(n, nrhs, seed=n)
    Xh, Xl, piv, st = mp.gesv_dd(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda())
    assert st["info_fp64"] == 0 and st["flags"] == 0 and st["iter"] >= 1, st
    Xh, Xl = Xh.cpu().numpy().reshape(n, nrhs), Xl.cpu().numpy().reshape(n, nrhs)
    r = orc.gesv_dd(A, B)
    assert r["info"] == 0
    kappa = orc.kappa_inf(A)
    # both are within ~kappa u_dd of the exact solution; the hi parts agree to
    # FP64 rounding, so their difference is exact
    diff = (Xh - r["Xhi"]) + (Xl - r["Xlo"])
    assert np.max(np.abs(diff)) <= 100 * n * kappa * UDD * np.max(np.abs(r["Xhi"])), (np.max(np.abs(diff)), kappa)
    # and the FP64 backward error of the hi part is at the FP64 floor
    assert np.all(orc.bwd_err(A, Xh, B) <= 1e-15)


def test_dd_on_floating_point_hilbert_matrix(torch, mp):
    n = 10
    A = np.array([[1.0 / (i + j + 1) for j in range(n)] for i in range(n)], order="F")
    x_ex = exact.solve(exact.to_frac_matrix(A.tolist()), [Fraction(1)] * n)
    Xh, Xl, _, st = mp.gesv_dd(torch.from_numpy(A).cuda(), torch.from_numpy(np.ones(n)).cuda(), itermax=20)
    assert st["flags"] == 0, st
    x = [Fraction(float(h)) + Fraction(float(l)) for h, l in zip(Xh.cpu().numpy(), Xl.cpu().numpy())]
    xm = max(abs(v) for v in x_ex)
    assert max(abs(a - e) for a, e in zip(x, x_ex)) <= 1e-16 * xm


def test_dd_integer_system_is_exact(torch, mp):
    n = 300
    rng = np.random.default_rng(4)
    A = np.asfortranarray(rng.integers(-20, 21, (n, n)).astype(np.float64))
    A[np.diag_indices(n)] += 400.0
    xt = rng.integers(-1000, 1001, (n, 3)).astype(np.float64)
    B = np.asfortranarray(A @ xt)
    Xh, Xl, _, st = mp.gesv_dd(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda())
    assert st["flags"] == 0
    Xh, Xl = Xh.cpu().numpy(), Xl.cpu().numpy()
    assert np.array_equal(Xh, xt) and np.all(np.abs(Xl) <= 1e-20)


def test_dd_singular_reports_info(torch, mp):
    n = 50
    A = inputs.small_integer_matrix(n, seed=2)
    A[:, 9] = 0.0
    _, _, _, st = mp.gesv_dd(torch.from_numpy(A).cuda(), torch.from_numpy(np.ones(n)).cuda())
    assert st["info_fp64"] == 10
