"""The paper's Fig. 4 experiment (Section 4) on the batched solver: random
200 x 200 systems of prescribed condition number, classical refinement with at
most 30 corrections and no FP64 fallback.

While kappa * u_s < 1, the mean number of corrections to the FP64 floor stays
within Datta's prediction ceil(ln u64 / (ln u_s + ln kappa)) plus one (the
acceptance rule takes one correction past FP64 accuracy to see the floor) and
does not decrease as kappa grows; once kappa * u_s >> 1 no system converges.
The FP32 counts are also compared system by system with the oracle's
Algorithm 1 (FP32 factors) on the same matrices.
"""
import numpy as np
import pytest

from paper_0808_2794_gb300 import inputs

pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53
US = {"fp32": 2.0 ** -24, "fp16": 2.0 ** -11, "bf16": 2.0 ** -8}
FAIL = 2 | 4 | 64  # STALLED | LOWP_BREAKDOWN | NOT_CONVERGED


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


def _run(torch, mp, As, Bs, prec):
    dA = [torch.from_numpy(a).cuda() for a in As]
    dB = [torch.from_numpy(b).cuda() for b in Bs]
    plan = mp.BatchedPlan(dA, dB, prec=prec, itermax=30, allow_fallback=False).run()
    torch.cuda.synchronize()
    Xs = [x.cpu().numpy() for x in plan.results()[0]]
    return plan.iter.copy(), plan.flags.copy(), Xs


@pytest.mark.parametrize("prec,kappas,bad_kappa", [("fp32", (1e1, 1e3, 1e5), 1e9),
                                                   ("fp16", (1e1, 1e2), 1e6)])
def test_mean_corrections_follow_datta_prediction(torch, mp, orc, prec, kappas, bad_kappa):
    means = []
    fam = inputs.conditioned_batch_family(200, 50, tuple(kappas) + (bad_kappa,), seed=7)
    for kappa, As, Bs, Xs in fam:
        it, fl, X = _run(torch, mp, As, Bs, prec)
        if kappa == bad_kappa:
            assert np.all(fl & FAIL), (kappa, it, fl)  # kappa u_s >> 1: no convergence
            continue
        assert np.all(fl == 0), (kappa, fl)
        pred = int(np.ceil(np.log(U64) / (np.log(US[prec]) + np.log(kappa))))
        assert 1 <= it.mean() <= pred + 1, (kappa, it.mean(), pred)
        means.append(it.mean())
        # every converged system meets the backward-error bar (oracle residual)
        for a, b, x in zip(As[:5], Bs[:5], X[:5]):
            assert orc.bwd_err(a, x.reshape(-1, 1), b)[0] <= 1e-14
    assert all(a <= b + 1e-12 for a, b in zip(means, means[1:])), means


def test_fp32_counts_match_oracle_algorithm_1(torch, mp, orc):
    """The same 12 systems at kappa = 1e4 through the batched GPU solver and
    through the oracle's Algorithm 1 with FP32 factors: the corrections to the
    FP64 floor agree to within one (the two factorizations round differently)."""
    (kappa, As, Bs, Xs), = inputs.conditioned_batch_family(200, 12, (1e4,), seed=11)
    it, fl, X = _run(torch, mp, As, Bs, "fp32")
    assert np.all(fl == 0), fl
    for k, (a, b) in enumerate(zip(As, Bs)):
        r = orc.gesv_ir(a, b[:, 0], factor_prec=32, allow_fallback=False)
        assert r["flags"] == 0
        assert abs(int(it[k]) - r["iter"]) <= 1, (k, int(it[k]), r["iter"])
