"""GPU parity of the batched small-system solver (Algorithm 1 per system in
one persistent launch) against the CPU oracle.

Tolerances as for the single-system solve: every column bwd <= 1e-14 and
||x - x_oracle|| / ||x_oracle|| <= 10 kappa_inf(A) 2^-53; pivots bit-exact
on pivot-unambiguous matrices (FP32 factorization); a system solved inside a
batch gives bit-for-bit the result it gives alone (one CTA owns it, every
reduction has a fixed order).
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
    return torch.from_numpy(np.asfortranarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def _check(orc, A, B, X):
    X = X.reshape(B.shape)
    assert np.all(orc.bwd_err(A, X, B) <= 1e-14)
    ref = orc.gesv_ir(A, B, factor_prec=64)["X"].reshape(B.shape)
    kappa = orc.kappa_inf(A)
    fwd = np.max(np.abs(X - ref)) / np.max(np.abs(ref))
    assert fwd <= 10 * kappa * U64, (fwd, kappa)


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16"])
def test_batched_small_systems(torch, mp, orc, prec):
    As, Bs, _ = inputs.batched_systems(count=48, seed=1, nmin=1, nmax=512)
    Xs, piv, it, fl, info = mp.gesv_batched([dev(torch, a) for a in As], [dev(torch, b) for b in Bs], prec=prec)
    assert np.all(fl == 0), fl
    assert np.all(info == 0) and np.all(it >= 0)
    for A, B, X in zip(As, Bs, Xs):
        _check(orc, A, B, host(X))


def test_batched_equals_alone(torch, mp):
    As, Bs, _ = inputs.batched_systems(count=20, seed=2)
    dA = [dev(torch, a) for a in As]
    dB = [dev(torch, b) for b in Bs]
    Xs, piv, it, fl, _ = mp.gesv_batched(dA, dB, prec="bf16")
    for i in range(len(As)):
        X1, p1, it1, fl1, _ = mp.gesv_batched([dA[i]], [dB[i]], prec="bf16")
        assert np.array_equal(host(X1[0]), host(Xs[i]))
        assert np.array_equal(host(p1[0]), host(piv[i]))
        assert it1[0] == it[i] and fl1[0] == fl[i]


def _unambiguous(n, seed):
    rng = np.random.default_rng(seed)
    L0 = np.tril(rng.uniform(-0.5, 0.5, (n, n)) / np.sqrt(n), -1) + np.eye(n)
    U0 = (np.triu(rng.uniform(-1, 1, (n, n)), 1) / np.sqrt(n)
          + np.diag(rng.uniform(1, 2, n) * rng.choice([-1, 1], n)))
    perm = rng.permutation(n)
    A = np.empty((n, n))
    A[perm] = L0 @ U0
    return np.asfortranarray(A)


def test_batched_pivots_exact(torch, mp, orc):
    sizes = [1, 2, 31, 32, 33, 100, 257, 512]
    As = [_unambiguous(n, n) for n in sizes]
    Bs = [np.asfortranarray(np.ones((n, 1))) for n in sizes]
    Xs, piv, it, fl, info = mp.gesv_batched([dev(torch, a) for a in As], [dev(torch, b) for b in Bs])
    for A, p in zip(As, piv):
        _, ref, _ = orc.getrf(A, prec=32)
        assert np.array_equal(host(p), np.asarray(ref)), A.shape


def test_batched_edge_cases(torch, mp, orc):
    rng = np.random.default_rng(3)
    n = 40
    sing = rng.standard_normal((n, n))
    sing[:, 7] = 0.0  # an exact zero pivot in any arithmetic
    nanA = rng.standard_normal((n, n)) + n * np.eye(n)
    nanA[5, 6] = np.nan
    hilb = np.array([[1.0 / (i + j + 1) for j in range(10)] for i in range(10)])
    good = rng.standard_normal((512, 512)) + 512 * np.eye(512)
    As = [np.asfortranarray(a) for a in (sing, nanA, hilb, good, np.eye(3))]
    Bs = [np.asfortranarray(np.ones((a.shape[0], 2))) for a in As]
    Bs.append(np.zeros((0, 1)))
    As.append(np.zeros((0, 0)))
    Xs, piv, it, fl, info = mp.gesv_batched([dev(torch, a) for a in As], [dev(torch, b) for b in Bs])
    assert info[0] == 8 and fl[0] & mp.FLAG_FALLBACK         # singular: FP64 reports the zero pivot
    assert fl[1] & mp.FLAG_NONFINITE_INPUT                      # NaN input
    assert fl[2] & mp.FLAG_FALLBACK and it[2] == -1             # kappa u32 > 1
    assert np.all(orc.bwd_err(hilb, host(Xs[2]), Bs[2]) <= 1e-14)
    assert fl[3] == 0
    _check(orc, good, Bs[3], host(Xs[3]))
    assert fl[4] == 0 and it[4] == 0 and np.array_equal(host(Xs[4]), Bs[4])
    assert fl[5] == 0 and it[5] == 0


def test_batched_rejects_large_n(torch, mp):
    A = dev(torch, np.eye(513))
    with pytest.raises(mp.MpError):
        mp.gesv_batched([A], [dev(torch, np.ones((513, 1)))])


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_batched_config_size(torch, mp, orc, prec):
    """The full batch of 4096 uneven systems (n log-uniform in [16, 512],
    nrhs 1..4): every system's backward error is checked."""
    As, Bs, _ = inputs.batched_systems(count=4096, seed=0)
    Xs, piv, it, fl, info = mp.gesv_batched([dev(torch, a) for a in As], [dev(torch, b) for b in Bs], prec=prec)
    assert np.all(fl == 0) and np.all(it >= 0)
    for A, B, X in zip(As, Bs, Xs):
        assert np.all(orc.bwd_err(A, host(X).reshape(B.shape), B) <= 1e-14)


@pytest.mark.parametrize("nb", [8, 16])
def test_batched_every_panel_width(torch, mp, orc, nb):
    """Every panel width the autotuner can choose gives correct solutions:
    a batch of uneven systems solved with the schedule forced to one width."""
    As, Bs, Xs = inputs.batched_systems(count=40, seed=5, nmin=16, nmax=200)
    mp.set_batched_schedule([(mp.BATCH_MAX_N, nb)])
    try:
        Xo, piv, it, fl, info = mp.gesv_batched([torch.from_numpy(a).cuda() for a in As],
                                                [torch.from_numpy(b).cuda() for b in Bs])
    finally:
        mp.set_batched_schedule(None)
    assert np.all(fl == 0) and np.all(it >= 0), (it, fl)
    for a, b, x, p in zip(As, Bs, Xo, piv):
        xh = x.cpu().numpy().reshape(a.shape[0], -1)
        assert np.all(orc.bwd_err(a, xh, b) <= 1e-14)
        ph = p.cpu().numpy()
        assert np.all((ph >= np.arange(1, a.shape[0] + 1)) & (ph <= a.shape[0]))
