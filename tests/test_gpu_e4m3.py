"""GPU parity of the FP8 (E4M3) rung of the trailing update (tcgen05
kind::f8f6f4): every 128 x 128 block of each operand (L21 by row block and
K-block, U12 by K-block and column block) is scaled by its own power of two so
that the block's largest magnitude lies below 2^8, rounded to E4M3 (round to
nearest even, saturating at 448), multiplied with FP32 accumulation, and each
K-block's product unscaled by its two blocks' scales.  The reference rounds
the same exactly scaled values with the oracle's E4M3 rounding (pinned by
brute force over all codes), so the only difference is the order of the FP32
sums: (K + 2) u32 |L8| |U8| + |C|.
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


def _block_round(orc, X):
    """X with every 128 x 128 block rounded to E4M3 at its own power-of-two
    scale 2^(8 - e), max |block| < 2^e (a zero block: 2^8), then unscaled."""
    out = np.empty_like(X)
    for r0 in range(0, X.shape[0], 128):
        for c0 in range(0, X.shape[1], 128):
            blk = X[r0:r0 + 128, c0:c0 + 128]
            m = float(np.max(np.abs(blk)))
            e = np.frexp(m)[1] if m > 0 else 0  # m < 2^e
            sc = 2.0 ** (8 - e)
            out[r0:r0 + 128, c0:c0 + 128] = orc.round_to(blk * sc, "e4m3") / sc
    return out


def _check(torch, mp, orc, L, U, C):
    M, K = L.shape
    N = U.shape[1]
    ld = lambda c: (c + 3) // 4 * 4
    Lt = torch.zeros((M, ld(K)), dtype=torch.float32, device="cuda")
    Ut = torch.zeros((K, ld(N)), dtype=torch.float32, device="cuda")
    Ct = torch.zeros((M, ld(N)), dtype=torch.float32, device="cuda")
    Lt[:, :K] = torch.from_numpy(L.astype(np.float32)).cuda()
    Ut[:, :N] = torch.from_numpy(U.astype(np.float32)).cuda()
    Ct[:, :N] = torch.from_numpy(C.astype(np.float32)).cuda()
    mp.lowp_gemm_update(Ct[:, :N], Lt[:, :K], Ut[:, :N], prec="e4m3")
    got = torch.Tensor.cpu(Ct).numpy()[:, :N].astype(np.float64)
    L32, U32_, C32 = (x.astype(np.float32).astype(np.float64) for x in (L, U, C))
    L8 = _block_round(orc, L32)
    U8 = _block_round(orc, U32_)
    ref = C32 - L8 @ U8
    bound = (K + 2) * U32 * (np.abs(L8) @ np.abs(U8) + np.abs(C32))
    assert np.all(np.abs(got - ref) <= bound)
    return got, ref


@pytest.mark.parametrize("M,N,K", [(256, 128, 64), (300, 200, 100), (1000, 777, 512), (129, 1025, 33)])
def test_trailing_update_e4m3(torch, mp, orc, M, N, K):
    rng = np.random.default_rng(M * 7 + N + K)
    L = rng.uniform(-1, 1, (M, K))
    U = rng.standard_normal((K, N)) * 3
    C = rng.standard_normal((M, N))
    _check(torch, mp, orc, L, U, C)


def test_trailing_update_e4m3_blocks_of_different_magnitude(torch, mp, orc):
    """Blocks whose magnitudes differ by 2^-20: each keeps E4M3's relative
    precision at its own scale (one scale per operand would flush the small
    blocks to zero), and K-blocks, row blocks and column blocks all differ."""
    M, N, K = 384, 300, 384
    rng = np.random.default_rng(3)
    L = rng.uniform(-1, 1, (M, K))
    U = rng.standard_normal((K, N))
    L[128:256, :] *= 2.0 ** -20
    L[:, 256:] *= 2.0 ** -12
    U[128:256, :] *= 2.0 ** 10
    U[:, 128:] *= 2.0 ** -16
    C = rng.standard_normal((M, N)) * 1e-3
    got, ref = _check(torch, mp, orc, L, U, C)
    # rows 128..255: with per-block scales their product keeps E4M3's relative
    # precision; one power-of-two scale per operand would round those entries
    # of L below E4M3's smallest subnormal, i.e. to zero
    L32, U32_, C32 = (x.astype(np.float32).astype(np.float64) for x in (L, U, C))

    def one_scale(X):
        e = np.frexp(float(np.max(np.abs(X))))[1]
        return orc.round_to(X * 2.0 ** (8 - e), "e4m3") / 2.0 ** (8 - e)
    exact = (L32 @ U32_)[128:256]
    err_block = np.max(np.abs((C32 - got)[128:256] - exact))
    err_one = np.max(np.abs((one_scale(L32) @ one_scale(U32_))[128:256] - exact))
    assert err_one >= 0.9 * np.max(np.abs(exact))  # flushed
    assert err_block <= 0.25 * err_one, (err_block, err_one)


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
