"""GPU parity of least squares by refinement of the augmented system
(Section 6 extension): the (m + n)-order system [alpha I, A; A^T, 0] solved by
the mixed-precision driver, against the oracle's FP64 solve of the same
system (the same alpha rule): x and r within 10 kappa_inf(K) u64, the
residual orthogonal to the columns of A."""
import numpy as np
import pytest

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


def _problem(m, n, nrhs, seed):
    rng = np.random.default_rng(seed)
    A = np.asfortranarray(rng.standard_normal((m, n)))
    B = np.asfortranarray(rng.standard_normal((m, nrhs)))
    return A, B


@pytest.mark.parametrize("m,n,nrhs,prec", [(12, 5, 1, "fp32"), (300, 100, 2, "fp32"), (700, 300, 1, "fp16x3"),
                                           (513, 511, 3, "bf16")])
def test_gels_matches_oracle(torch, mp, orc, m, n, nrhs, prec):
    A, B = _problem(m, n, nrhs, seed=m + n)
    X, R, st = mp.gels(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), prec=prec, refine="auto")
    assert st["info_fp64"] == 0 and st["bwd_err"] <= 1e-14, st
    X, R = X.cpu().numpy().reshape(n, nrhs), R.cpu().numpy().reshape(m, nrhs)
    ref = orc.gels_aug(A, B)
    alpha = ref["alpha"]
    K = np.zeros((m + n, m + n))
    K[:m, :m] = alpha * np.eye(m)
    K[:m, m:] = A
    K[m:, :m] = A.T
    kappa = orc.kappa_inf(np.asfortranarray(K))
    Y = np.vstack([R / alpha, X])
    Yr = np.vstack([ref["R"] / alpha, ref["X"]])
    assert np.max(np.abs(Y - Yr)) <= 10 * kappa * U64 * np.max(np.abs(Yr))
    assert np.max(np.abs(A.T @ R)) <= 1e-10 * np.max(np.abs(A)) * np.max(np.abs(R)) * m
    assert np.allclose(R, B - A @ X, rtol=0, atol=1e-9 * np.max(np.abs(B)))


def test_gels_square_is_a_solve(torch, mp, orc):
    n = 200
    A, B = _problem(n, n, 1, seed=9)
    X, R, st = mp.gels(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda())
    x = X.cpu().numpy().reshape(n, 1)
    ref = orc.gesv_ir(A, B, factor_prec=64)["X"].reshape(n, 1)
    assert np.max(np.abs(x - ref)) <= 1e-9 * np.max(np.abs(ref))
    assert np.max(np.abs(R.cpu().numpy())) <= 1e-10 * np.max(np.abs(B))


def test_gels_rejects_bad_shapes(torch, mp):
    A = torch.zeros((3, 5), dtype=torch.float64, device="cuda")
    with pytest.raises(mp.MpError):
        mp.gels(A, torch.zeros(3, dtype=torch.float64, device="cuda"))
