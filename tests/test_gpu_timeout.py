"""Failure detection without a GPU fault: every device-side wait of the
library is bounded, and a wait that runs out records MP_FLAG_TIMEOUT and the
site, and the kernel returns.  Each test runs one of the library's own
bounded waits (the triangular solves' grid barrier, the panel kernel's and the
tensor-core kernels' mbarrier waits) on a condition nothing satisfies, with a
20 ms limit, then checks the recorded status, that the call came back within
a second, and that the context still solves a system correctly."""
import time

import numpy as np
import pytest

from paper_0808_2794_gb300 import inputs

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("site", [2, 3, 4])
def test_bounded_wait_gives_up_and_reports(torch, mp, orc, site):
    t0 = time.perf_counter()
    flags, where, passed = mp.selftest_wait_timeout(site, 20_000_000)
    dt = time.perf_counter() - t0
    assert flags & mp.FLAG_TIMEOUT, flags
    assert where == site
    assert passed == 0  # no CTA got past a barrier that could not complete
    assert dt < 1.0, dt
    # the context is still usable: a solve right after is correct
    A, B, _ = inputs.dense_system(96, nrhs=2, seed=site)
    X, _, st = mp.gesv(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda())
    assert st["flags"] == 0
    assert np.all(orc.bwd_err(A, X.cpu().numpy(), B) <= 1e-14)


def test_selftest_rejects_bad_arguments(torch, mp):
    with pytest.raises(mp.MpError):
        mp.selftest_wait_timeout(1, 1000)
    with pytest.raises(mp.MpError):
        mp.selftest_wait_timeout(2, 0)
