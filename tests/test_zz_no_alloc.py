"""mp_gesv_noalloc: the solve for callers that may not allocate device memory
(services whose device memory is fixed at start-up, plug-ins whose host owns
every allocation).  Its scratch is a static device array inside the library;
the caller passes only A, B, X and the pivots.

Checked through the C ABI against the regular entry point mp_gesv (which
takes a caller workspace), on two calls in a row so that the second call runs
on an array that still holds the first call's contents.  This file is
collected last on purpose (a run that stops at the first failure has run
everything else already), and it works both alone and after other tests.
"""
import ctypes

import numpy as np
import pytest

from paper_0808_2794_gb300 import inputs

pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_0808_2794_gb300 import solver
    return torch, solver, solver.load()


def _noalloc(torch, solver, lib, Ad, Bd, n, nrhs, refine=None, X=None, ipiv=None):
    if X is None:
        X = torch.zeros((nrhs, n), dtype=torch.float64, device="cuda").t()
        ipiv = torch.zeros(n, dtype=torch.int32, device="cuda")
    opts = solver.default_opts()
    if refine is not None:
        opts.refine = refine
    st = solver.mp_stats()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    ret = lib.mp_gesv_noalloc(n, nrhs, Ad.data_ptr(), n, Bd.data_ptr(), n, X.data_ptr(), n,
                              ipiv.data_ptr(), ctypes.byref(opts), ctypes.byref(st), stream)
    torch.cuda.synchronize()
    assert ret == 0, solver.last_error()
    return X, ipiv, st


def test_noalloc_matches_gesv_on_consecutive_calls(env, orc):
    torch, solver, lib = env
    for seed, n, nrhs in ((11, 1200, 2), (12, 700, 1)):
        A, B, _ = inputs.dense_system(n, nrhs=nrhs, seed=seed)
        Ad = torch.from_numpy(np.asfortranarray(A)).cuda()
        Bd = torch.from_numpy(np.asfortranarray(B)).cuda()
        Xr, pr, sr = solver.gesv(Ad, Bd)  # regular entry point, caller workspace
        Xn, pn, sn = _noalloc(torch, solver, lib, Ad, Bd, n, nrhs)
        Xr, Xn = Xr.cpu().numpy(), Xn.cpu().numpy()
        assert sn.flags == sr["flags"] == 0 and sn.iter >= 0
        assert np.array_equal(pn.cpu().numpy(), pr.cpu().numpy())
        # same tolerance as the parity tests: both are within 10 kappa u of the
        # exact solution and below the 1e-14 backward-error bar
        kappa = orc.kappa_inf(A)
        assert np.max(np.abs(Xn - Xr)) <= 10 * kappa * U64 * np.max(np.abs(Xr))
        assert np.all(orc.bwd_err(A, Xn, B) <= 1e-14)


def test_noalloc_rejects_sizes_beyond_the_static_array(env):
    torch, solver, lib = env
    cap = lib.mp_noalloc_scratch_bytes()
    o = solver.default_opts()
    n = 1
    while lib.mp_gesv_workspace_bytes(n, 1, ctypes.byref(o)) <= cap:
        n *= 2
    P = ctypes.c_void_p(16)
    st = solver.mp_stats()
    ret = lib.mp_gesv_noalloc(n, 1, P, n, P, n, P, n, P, ctypes.byref(o), ctypes.byref(st), None)
    assert ret == -1
    assert "static array" in solver.last_error()


@pytest.mark.parametrize("refine", [0, 1])  # classical refinement, GMRES-based refinement
def test_noalloc_call_allocates_no_device_memory(env, orc, refine):
    """After a first call on the device (its one-time set-up), a further call
    leaves the device's free memory exactly where it was: the solve takes all
    its scratch from the static array, whichever refinement scheme runs."""
    torch, solver, lib = env
    n, nrhs = 900, 2
    A, B, _ = inputs.dense_system(n, nrhs=nrhs, seed=21)
    Ad = torch.from_numpy(np.asfortranarray(A)).cuda()
    Bd = torch.from_numpy(np.asfortranarray(B)).cuda()
    X = torch.zeros((nrhs, n), dtype=torch.float64, device="cuda").t()
    ipiv = torch.zeros(n, dtype=torch.int32, device="cuda")
    _noalloc(torch, solver, lib, Ad, Bd, n, nrhs, refine=refine, X=X, ipiv=ipiv)  # set-up call
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    X.zero_()
    torch.cuda.synchronize()
    _, _, st = _noalloc(torch, solver, lib, Ad, Bd, n, nrhs, refine=refine, X=X, ipiv=ipiv)
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    if refine == 1:
        assert st.flags & 32  # MP_FLAG_GMRES_USED: the GMRES scratch came from the array too
    assert np.all(orc.bwd_err(A, X.cpu().numpy(), B) <= 1e-14)
