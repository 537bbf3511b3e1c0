"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/mpsolve.h; argument checking happens before any device
work (so these run without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mpsolve.h")).read()
    return sorted(set(re.findall(r"MP_API\s+[\w\s\*]*?\b(mp_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_0808_2794_gb300 import solver
    return solver.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 14
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_header():
    from paper_0808_2794_gb300 import solver
    assert sorted(solver.exported_symbols()) == _declared()


def test_argument_errors_are_lapack_style(lib):
    from paper_0808_2794_gb300 import solver
    o = solver.default_opts()
    st = solver.mp_stats()
    P = ctypes.c_void_p(0)
    # n < 0 -> -1
    assert lib.mp_gesv(-1, 1, P, 1, P, 1, P, 1, P, P, 0, ctypes.byref(o), ctypes.byref(st), P) == -1
    # nrhs > 8 -> -2
    assert lib.mp_gesv(4, 9, P, 4, P, 4, P, 4, P, P, 0, ctypes.byref(o), ctypes.byref(st), P) == -2
    # lda < n -> -4 (checked before any pointer is used)
    dummy = ctypes.c_void_p(16)
    assert lib.mp_gesv(4, 1, dummy, 3, dummy, 4, dummy, 4, dummy, dummy, 1 << 30,
                       ctypes.byref(o), ctypes.byref(st), P) == -4
    # workspace too small -> -11
    assert lib.mp_gesv(4, 1, dummy, 4, dummy, 4, dummy, 4, dummy, dummy, 16,
                       ctypes.byref(o), ctypes.byref(st), P) == -11
    assert "workspace" in solver.last_error()
    # invalid options -> -12
    bad = solver.default_opts(itermax=-1)
    assert lib.mp_gesv(4, 1, dummy, 4, dummy, 4, dummy, 4, dummy, dummy, 1 << 30,
                       ctypes.byref(bad), ctypes.byref(st), P) == -12
    # n == 0 is a successful no-op
    assert lib.mp_gesv(0, 1, P, 1, P, 1, P, 1, P, P, 0, ctypes.byref(o), ctypes.byref(st), P) == 0


def test_workspace_queries_scale(lib):
    from paper_0808_2794_gb300 import solver
    o = solver.default_opts()
    w1 = lib.mp_gesv_workspace_bytes(1024, 1, ctypes.byref(o))
    w2 = lib.mp_gesv_workspace_bytes(2048, 1, ctypes.byref(o))
    # dominated by the n^2 working matrix (FP64 room for the fallback) and the
    # inverted diagonal blocks of the factors (n x BI per triangle)
    assert 8 * 1024 * 1024 <= w1 < 32 * 1024 * 1024
    assert 2.5 < w2 / w1 < 4.5
    o.allow_fallback = 0
    assert lib.mp_gesv_workspace_bytes(2048, 1, ctypes.byref(o)) < w2 * 0.75
    assert lib.mp_factor_ld(1) == 32 and lib.mp_factor_ld(33) == 64


def test_batched_schedule_set_get_and_validation():
    """The batched solver's tile schedule (host-side state, no GPU needed):
    replaced, read back, validated and restored."""
    from paper_0808_2794_gb300 import solver
    base = solver.batched_schedule()
    assert base and base[-1][0] >= solver.BATCH_MAX_N
    assert all(nb in (8, 16) for _, nb in base)
    try:
        solver.set_batched_schedule([(64, 8), (512, 16)])
        assert solver.batched_schedule() == [(64, 8), (512, 16)]
        for bad in ([(64, 12), (512, 16)], [(128, 16), (64, 16)], [(256, 16)]):
            with pytest.raises(solver.MpError):
                solver.set_batched_schedule(bad)
        assert solver.batched_schedule() == [(64, 8), (512, 16)]
    finally:
        solver.set_batched_schedule(None)
    assert solver.batched_schedule() == base
