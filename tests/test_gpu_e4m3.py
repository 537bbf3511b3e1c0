"""GPU parity of the FP8 (E4M3) rung of the trailing update (tcgen05
kind::f8f6f4): each operand is scaled by a power of two so that its largest
magnitude lies below 2^8, rounded to E4M3 (round to nearest even, saturating
at 448), multiplied with FP32 accumulation, and the product unscaled in the
epilogue.  The reference rounds the same exactly scaled values with the
oracle's E4M3 rounding (pinned by brute force over all codes), so the only
difference is the order of the FP32 sums: (K + 2) u32 |L8| |U8| + |C|.
"""
import numpy as np
import pytest

from paper_0808_2794_gb300 import inputs

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
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


def _scale(x):
    m = float(np.max(np.abs(x)))
    e = np.frexp(m)[1] if m > 0 else 0  # m < 2^e
    return 2.0 ** (8 - e)


@pytest.mark.parametrize("M,N,K", [(256, 128, 64), (300, 200, 100), (1000, 777, 512), (129, 1025, 33)])
def test_trailing_update_e4m3(torch, mp, orc, M, N, K):
    rng = np.random.default_rng(M * 7 + N + K)
    ld = lambda c: (c + 3) // 4 * 4
    L = rng.uniform(-1, 1, (M, K))
    U = rng.standard_normal((K, N)) * 3
    C = rng.standard_normal((M, N))
    Lt = torch.zeros((M, ld(K)), dtype=torch.float32, device="cuda")
    Ut = torch.zeros((K, ld(N)), dtype=torch.float32, device="cuda")
    Ct = torch.zeros((M, ld(N)), dtype=torch.float32, device="cuda")
    Lt[:, :K] = torch.from_numpy(L.astype(np.float32)).cuda()
    Ut[:, :N] = torch.from_numpy(U.astype(np.float32)).cuda()
    Ct[:, :N] = torch.from_numpy(C.astype(np.float32)).cuda()
    mp.lowp_gemm_update(Ct[:, :N], Lt[:, :K], Ut[:, :N], prec="e4m3")
    got = torch.Tensor.cpu(Ct).numpy()[:, :N].astype(np.float64)
    L32, U32_, C32 = (x.astype(np.float32).astype(np.float64) for x in (L, U, C))
    sl, su = _scale(L32), _scale(U32_)
    L8 = orc.round_to(L32 * sl, "e4m3") / sl
    U8 = orc.round_to(U32_ * su, "e4m3") / su
    ref = C32 - L8 @ U8
    bound = (K + 2) * U32 * (np.abs(L8) @ np.abs(U8) + np.abs(C32))
    assert np.all(np.abs(got - ref) <= bound)


def test_gesv_e4m3_with_gmres(torch, mp, orc):
    """u = 2^-4: the factorization is a coarse preconditioner; GMRES-based
    refinement (Section 2.2) still reaches FP64 accuracy on a well
    conditioned system without the FP64 fallback."""
    n = 1024
    A, B, _ = inputs.conditioned_system(n, 4.0, seed=6)
    X, _, st = mp.gesv(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), prec="e4m3", nb_outer=128,
                       refine="auto")
    assert not st["flags"] & mp.FLAG_FALLBACK, st
    X = X.cpu().numpy().reshape(n, 1)
    assert np.all(orc.bwd_err(A, X, B) <= 1e-14)
    ref = orc.gesv_ir(A, B, factor_prec=64)["X"].reshape(n, 1)
    assert np.max(np.abs(X - ref)) / np.max(np.abs(ref)) <= 10 * orc.kappa_inf(A) * U64
