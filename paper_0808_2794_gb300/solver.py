"""Thin Python binding of the C ABI in ``include/mpsolve.h``.

Argument marshalling only: every step of the solve runs in the CUDA library
``_build/libmpsolve.so`` (built by ``paper_0808_2794_gb300.build``).  There is
no CPU fallback: if the library or a GPU is missing, these functions raise.

Matrices are column-major (LAPACK layout).  A torch tensor ``A`` of shape
(n, n) is column-major when ``A.stride() == (1, lda)``; ``colmajor(t)`` returns
such a copy.  Workspace comes from PyTorch's caching allocator.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

PREC = {"fp32": 0, "fp16x3": 1, "bf16": 2, "fp16": 3, "e4m3": 4, "fp64": 5}
REFINE = {"classical": 0, "gmres": 1, "auto": 2}

FLAG_FALLBACK = 1
FLAG_STALLED = 2
FLAG_LOWP_BREAKDOWN = 4
FLAG_NONFINITE_INPUT = 8
FLAG_TIMEOUT = 16
FLAG_GMRES_USED = 32
FLAG_NOT_CONVERGED = 64


class mp_opts(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int), ("refine", ctypes.c_int), ("itermax", ctypes.c_int),
                ("tol", ctypes.c_double), ("gmres_restart", ctypes.c_int),
                ("gmres_tol", ctypes.c_double), ("stall_ratio", ctypes.c_double),
                ("allow_fallback", ctypes.c_int), ("nb_outer", ctypes.c_int),
                ("nb_inner", ctypes.c_int)]


class mp_stats(ctypes.Structure):
    _fields_ = [("iter", ctypes.c_int), ("flags", ctypes.c_uint), ("info", ctypes.c_int),
                ("n_precond", ctypes.c_int), ("bwd_err", ctypes.c_double), ("nhist", ctypes.c_int),
                ("hist", ctypes.c_double * 32), ("ms_convert", ctypes.c_float),
                ("ms_factor", ctypes.c_float), ("ms_refine", ctypes.c_float),
                ("ms_fallback", ctypes.c_float)]

    def as_dict(self):
        return dict(iter=self.iter, flags=self.flags, info=self.info, n_precond=self.n_precond,
                    bwd_err=self.bwd_err, hist=list(self.hist[: self.nhist]),
                    ms_convert=self.ms_convert, ms_factor=self.ms_factor,
                    ms_refine=self.ms_refine, ms_fallback=self.ms_fallback)


class mp_sparse_opts(ctypes.Structure):
    _fields_ = [("m_out", ctypes.c_int), ("m_in", ctypes.c_int), ("inner", ctypes.c_int),
                ("max_cycles", ctypes.c_int), ("tol", ctypes.c_double)]


class mp_sparse_stats(ctypes.Structure):
    _fields_ = [("cycles", ctypes.c_int), ("outer_steps", ctypes.c_int), ("inner_steps", ctypes.c_int),
                ("flags", ctypes.c_uint), ("bwd_err", ctypes.c_double), ("nhist", ctypes.c_int),
                ("hist", ctypes.c_double * 32)]

    def as_dict(self):
        return dict(cycles=self.cycles, outer_steps=self.outer_steps, inner_steps=self.inner_steps,
                    flags=self.flags, bwd_err=self.bwd_err, hist=list(self.hist[: self.nhist]))


INNER = {"fp32": 0, "fp64": 1, "none": 2}

_lib = None
_lock = threading.Lock()

_P = ctypes.c_void_p
_I = ctypes.c_int
_Z = ctypes.c_size_t
_SIGS = {
    "mp_default_opts": (None, [ctypes.POINTER(mp_opts)]),
    "mp_last_error": (ctypes.c_char_p, []),
    "mp_gesv_workspace_bytes": (_Z, [_I, _I, ctypes.POINTER(mp_opts)]),
    "mp_gesv": (_I, [_I, _I, _P, _I, _P, _I, _P, _I, _P, _P, _Z, ctypes.POINTER(mp_opts),
                     ctypes.POINTER(mp_stats), _P]),
    "mp_gesv_host_workspace_bytes": (_Z, [_I, _I, ctypes.POINTER(mp_opts)]),
    "mp_gesv_host": (_I, [_I, _I, _P, _I, _P, _I, _P, _I, _P, _P, _Z, ctypes.POINTER(mp_opts),
                          ctypes.POINTER(mp_stats), _P]),
    "mp_posv_workspace_bytes": (_Z, [_I, _I, ctypes.POINTER(mp_opts)]),
    "mp_posv": (_I, [_I, _I, _P, _I, _P, _I, _P, _I, _P, _Z, ctypes.POINTER(mp_opts),
                     ctypes.POINTER(mp_stats), _P]),
    "mp_gesv_adjoint_workspace_bytes": (_Z, [_I, ctypes.POINTER(mp_opts)]),
    "mp_gesv_adjoint": (_I, [_I, _I, _P, _I, _P, _I, _P, _I, _P, _I, _P, _I, _P, _Z, _P, _Z,
                             ctypes.POINTER(mp_opts), ctypes.POINTER(mp_stats), _P]),
    "mp_gesv_batched_workspace_bytes": (_Z, [_I, _P, _P, ctypes.POINTER(mp_opts)]),
    "mp_gesv_batched": (_I, [_I, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _Z,
                             ctypes.POINTER(mp_opts), _P]),
    "mp_factor_ld": (_I, [_I]),
    "mp_getrf_workspace_bytes": (_Z, [_I, ctypes.POINTER(mp_opts)]),
    "mp_convert": (_I, [_I, _P, _I, _P, _I, _P, _P, _P, _Z, _P]),
    "mp_getrf_lowp": (_I, [_I, _P, _I, _P, ctypes.POINTER(mp_opts), _P, _Z,
                           ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_uint32), _P]),
    "mp_potrf_lowp": (_I, [_I, _P, _I, ctypes.POINTER(mp_opts), _P, _Z,
                           ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_uint32), _P]),
    "mp_getrs_workspace_bytes": (_Z, [_I, _I]),
    "mp_getrs_lowp": (_I, [_I, _I, _P, _I, _P, _P, _I, _P, _I, _P, _Z, _P]),
    "mp_residual_workspace_bytes": (_Z, [_I, _I]),
    "mp_lowp_gemm_workspace_bytes": (_Z, [_I, _I, _I, _I]),
    "mp_lowp_gemm_update": (_I, [_I, _I, _I, _I, _P, _I, _P, _I, _P, _I, _P, _Z, _P]),
    "mp_residual": (_I, [_I, _I, _P, _I, _P, _I, _P, _I, _P, _I, _P, _Z, _P]),
    "mp_noalloc_scratch_bytes": (_Z, []),
    "mp_gesv_noalloc": (_I, [_I, _I, _P, _I, _P, _I, _P, _I, _P, ctypes.POINTER(mp_opts),
                             ctypes.POINTER(mp_stats), _P]),
    "mp_batched_set_schedule": (_I, [_I, _P, _P]),
    "mp_batched_get_schedule": (_I, [_I, ctypes.POINTER(ctypes.c_int), _P, _P]),
    "mp_gesv_dd_workspace_bytes": (_Z, [_I, _I]),
    "mp_gesv_dd": (_I, [_I, _I, _P, _I, _P, _I, _P, _P, _I, _P, _I, _P, _Z, ctypes.POINTER(mp_stats), _P]),
    "mp_gels_workspace_bytes": (_Z, [_I, _I, _I, ctypes.POINTER(mp_opts)]),
    "mp_gels": (_I, [_I, _I, _I, _P, _I, _P, _I, _P, _I, _P, _I, ctypes.c_double, _P, _Z, ctypes.POINTER(mp_opts),
                     ctypes.POINTER(mp_stats), _P]),
    "mp_sparse_default_opts": (None, [ctypes.POINTER(mp_sparse_opts)]),
    "mp_fgmres_workspace_bytes": (_Z, [_I, ctypes.c_longlong, ctypes.POINTER(mp_sparse_opts)]),
    "mp_fgmres": (_I, [_I, ctypes.c_longlong, _P, _P, _P, _P, _P, _P, _Z, ctypes.POINTER(mp_sparse_opts),
                       ctypes.POINTER(mp_sparse_stats), _P]),
    "mp_sparse_gmres_cycle": (_I, [_I, ctypes.c_longlong, _P, _P, _P, _P, _P, _I, _I, _P, _Z,
                                   ctypes.POINTER(ctypes.c_int), _P]),
    "mp_csr_spmv": (_I, [_I, ctypes.c_longlong, _P, _P, _P, _P, _P, _I, _P]),
    "mp_selftest_workspace_bytes": (_Z, []),
    "mp_selftest_wait_timeout": (_I, [_I, ctypes.c_ulonglong, _P, _Z, ctypes.POINTER(ctypes.c_uint),
                                      ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), _P]),
    "mp_profile_enable": (None, [ctypes.c_uint]),
    "mp_profile_sample": (None, [ctypes.c_int]),
    "mp_profile_collect": (_I, [_P, _P, _P]),
    "mp_launch_count": (ctypes.c_longlong, []),
}

KERNEL_CLASSES = ["panel", "rowmoves", "trsm", "update", "panelgemm", "trsv", "residual"]


def profile_enable(classes=()):
    """Time the named kernel classes with CUDA events (empty: off, clears records)."""
    mask = 0
    for c in classes:
        mask |= 1 << KERNEL_CLASSES.index(c)
    load().mp_profile_enable(mask)


def profile_sample(every=1):
    """Time one launch in every `every` of each enabled class (1: all)."""
    load().mp_profile_sample(int(every))


def profile_collect():
    """{class: (ms, launches, work)} for the records since profile_enable."""
    import numpy as np
    ms = np.zeros(len(KERNEL_CLASSES))
    ln = np.zeros(len(KERNEL_CLASSES), dtype=np.int64)
    wk = np.zeros(len(KERNEL_CLASSES))
    _check(load().mp_profile_collect(ms.ctypes.data, ln.ctypes.data, wk.ctypes.data),
           "mp_profile_collect")
    return {c: (float(ms[i]), int(ln[i]), float(wk[i])) for i, c in enumerate(KERNEL_CLASSES)}


def launch_count() -> int:
    return int(load().mp_launch_count())


def exported_symbols():
    """Names of the C ABI entry points this binding expects."""
    return sorted(_SIGS)


def load(build_if_missing: bool = True):
    """Load libmpsolve.so (building it with nvcc if needed); raises if impossible."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                if not build_if_missing:
                    raise RuntimeError(f"CUDA library not built: {path}")
                path = _build.build()
            lib = ctypes.CDLL(path)
            for name, (res, args) in _SIGS.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def last_error() -> str:
    return load().mp_last_error().decode()


def default_opts(**kw) -> mp_opts:
    o = mp_opts()
    load().mp_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if k == "prec" and isinstance(v, str):
            v = PREC[v]
        if k == "refine" and isinstance(v, str):
            v = REFINE[v]
        setattr(o, k, v)
    return o


class MpError(RuntimeError):
    pass


def _check(ret, what):
    if ret < 0:
        raise MpError(f"{what} returned {ret}: {last_error()}")
    return ret


# ---------------------------------------------------------------- torch helpers
def _torch():
    import torch
    if not torch.cuda.is_available():
        raise MpError("a CUDA device is required (there is no CPU path)")
    return torch


def colmajor(t):
    """Column-major (Fortran-order) copy of a 2-D tensor (view if already)."""
    if t.dim() == 1:
        t = t.reshape(-1, 1)
    if t.stride(0) == 1 and t.stride(1) >= max(1, t.shape[0]):
        return t
    return t.t().contiguous().t()


def _ld(t):
    """Leading dimension of a column-major 2-D tensor (any value >= rows for one column)."""
    return t.stride(1) if t.shape[1] > 1 else max(1, t.shape[0], t.stride(1))


def _stream_ptr(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def workspace(nbytes: int, device=None):
    torch = _torch()
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device or "cuda")


def gesv(A, B, prec="fp32", refine="classical", itermax=30, tol=1e-14, allow_fallback=True,
         nb_outer=0, gmres_restart=30, gmres_tol=1e-6, work=None, stream=None):
    """Solve A X = B (Algorithm 1).  A: (n, n) float64 CUDA tensor, B: (n,) or
    (n, nrhs).  Returns (X, ipiv, stats) with X column-major float64 and ipiv
    int32 (LAPACK 1-based)."""
    torch = _torch()
    lib = load()
    A = colmajor(A)
    squeeze = B.dim() == 1
    B = colmajor(B)
    n, nrhs = B.shape
    opts = default_opts(prec=prec, refine=refine, itermax=itermax, tol=tol,
                        allow_fallback=int(bool(allow_fallback)), nb_outer=nb_outer,
                        gmres_restart=gmres_restart, gmres_tol=gmres_tol)
    X = torch.empty((nrhs, n), dtype=torch.float64, device=A.device).t()
    ipiv = torch.empty(max(n, 1), dtype=torch.int32, device=A.device)
    need = lib.mp_gesv_workspace_bytes(n, nrhs, ctypes.byref(opts))
    if work is None or work.numel() < need:
        work = workspace(need, A.device)
    st = mp_stats()
    ret = lib.mp_gesv(n, nrhs, A.data_ptr(), _ld(A), B.data_ptr(), _ld(B), X.data_ptr(),
                      _ld(X), ipiv.data_ptr(), work.data_ptr(), work.numel(),
                      ctypes.byref(opts), ctypes.byref(st), _stream_ptr(stream))
    _check(ret, "mp_gesv")
    d = st.as_dict()
    d["info_fp64"] = ret
    return (X[:, 0] if squeeze else X), ipiv[:n], d


def posv(A, B, prec="fp32", refine="classical", itermax=30, tol=1e-14, allow_fallback=True,
         nb_outer=0, gmres_restart=30, gmres_tol=1e-6, work=None, stream=None):
    """Solve A X = B for symmetric positive definite A from its lower triangle
    (Cholesky variant).  Returns (X, stats); stats["info_fp64"] > 0 when A is
    not positive definite."""
    torch = _torch()
    lib = load()
    A = colmajor(A)
    squeeze = B.dim() == 1
    B = colmajor(B)
    n, nrhs = B.shape
    opts = default_opts(prec=prec, refine=refine, itermax=itermax, tol=tol,
                        allow_fallback=int(bool(allow_fallback)), nb_outer=nb_outer,
                        gmres_restart=gmres_restart, gmres_tol=gmres_tol)
    X = torch.empty((nrhs, n), dtype=torch.float64, device=A.device).t()
    need = lib.mp_posv_workspace_bytes(n, nrhs, ctypes.byref(opts))
    if work is None or work.numel() < need:
        work = workspace(need, A.device)
    st = mp_stats()
    ret = lib.mp_posv(n, nrhs, A.data_ptr(), _ld(A), B.data_ptr(), _ld(B), X.data_ptr(), _ld(X),
                      work.data_ptr(), work.numel(), ctypes.byref(opts), ctypes.byref(st),
                      _stream_ptr(stream))
    _check(ret, "mp_posv")
    d = st.as_dict()
    d["info_fp64"] = ret
    return (X[:, 0] if squeeze else X), d


def gesv_adjoint(A, X, G, work, prec="fp32", allow_fallback=True, nb_outer=0, adj_work=None,
                 stream=None):
    """Bbar = A^{-T} G and Abar = -Bbar X^T from the factors a preceding gesv /
    posv call left in `work` (pass that call's workspace and options).
    Returns (Abar, Bbar, stats)."""
    torch = _torch()
    lib = load()
    A = colmajor(A)
    squeeze = G.dim() == 1
    G = colmajor(G)
    X = colmajor(X)
    n, nrhs = G.shape
    opts = default_opts(prec=prec, allow_fallback=int(bool(allow_fallback)), nb_outer=nb_outer)
    need = lib.mp_gesv_adjoint_workspace_bytes(n, ctypes.byref(opts))
    if adj_work is None or adj_work.numel() < need:
        adj_work = workspace(need, A.device)
    Bbar = torch.empty((nrhs, n), dtype=torch.float64, device=A.device).t()
    Abar = torch.empty((n, n), dtype=torch.float64, device=A.device).t()
    st = mp_stats()
    ret = lib.mp_gesv_adjoint(n, nrhs, A.data_ptr(), _ld(A), X.data_ptr(), _ld(X), G.data_ptr(), _ld(G),
                              Bbar.data_ptr(), _ld(Bbar), Abar.data_ptr(), max(n, 1),
                              work.data_ptr(), work.numel(), adj_work.data_ptr(), adj_work.numel(),
                              ctypes.byref(opts), ctypes.byref(st), _stream_ptr(stream))
    _check(ret, "mp_gesv_adjoint")
    return Abar, (Bbar[:, 0] if squeeze else Bbar), st.as_dict()


def _make_solve_fn():
    torch = _torch()

    class SolveFn(torch.autograd.Function):
        """X = A^{-1} B with mixed-precision refinement; backward through the
        adjoint solve with the same factors (Abar = -A^{-T} G X^T,
        Bbar = A^{-T} G)."""

        @staticmethod
        def forward(ctx, A, B, prec="fp32", nb_outer=0):
            work = workspace(load().mp_gesv_workspace_bytes(
                A.shape[0], 1 if B.dim() == 1 else B.shape[1],
                ctypes.byref(default_opts(prec=prec, nb_outer=nb_outer))), A.device)
            X, _, st = gesv(A.detach(), B.detach(), prec=prec, nb_outer=nb_outer, work=work)
            X = X.contiguous() if X.dim() == 1 else X
            ctx.save_for_backward(A, X)
            ctx.work, ctx.prec, ctx.nb_outer, ctx.vec = work, prec, nb_outer, B.dim() == 1
            return X.clone()

        @staticmethod
        def backward(ctx, G):
            A, X = ctx.saved_tensors
            Abar, Bbar, _ = gesv_adjoint(A.detach(), X, G.contiguous(), ctx.work, prec=ctx.prec,
                                         nb_outer=ctx.nb_outer)
            return Abar, Bbar, None, None

    return SolveFn


def solve_fn():
    """The torch.autograd.Function of the solve (built on first use)."""
    global _SOLVE_FN
    if _SOLVE_FN is None:
        _SOLVE_FN = _make_solve_fn()
    return _SOLVE_FN


_SOLVE_FN = None


BATCH_MAX_N = 512


class BatchedPlan:
    """Argument tables of one batch (host arrays of sizes and device pointers)
    prepared once, so that repeated solves of the same batch only make the C
    call.  Outputs X, ipiv are allocated here and reused by every run()."""

    def __init__(self, As, Bs, prec="fp32", itermax=30, tol=1e-14, allow_fallback=True):
        import numpy as np
        torch = _torch()
        self.lib = load()
        count = len(As)
        self.count = count
        self.A_c = [colmajor(a) for a in As]
        self.B_c = [colmajor(b) for b in Bs]
        self.vec = [b.dim() == 1 for b in Bs]
        self.n = np.array([a.shape[0] for a in self.A_c], dtype=np.int32)
        self.nrhs = np.array([b.shape[1] for b in self.B_c], dtype=np.int32)
        self.X_c = [torch.empty((int(r), int(m)), dtype=torch.float64, device=a.device).t()
                    for a, m, r in zip(self.A_c, self.n, self.nrhs)]
        self.piv = [torch.zeros(max(int(m), 1), dtype=torch.int32, device=a.device)
                    for a, m in zip(self.A_c, self.n)]
        self.lda = np.array([_ld(a) for a in self.A_c], dtype=np.int32)
        self.ldb = np.array([_ld(b) for b in self.B_c], dtype=np.int32)
        self.ldx = np.array([_ld(x) for x in self.X_c], dtype=np.int32)
        self.pa = np.array([a.data_ptr() for a in self.A_c], dtype=np.uint64)
        self.pb = np.array([b.data_ptr() for b in self.B_c], dtype=np.uint64)
        self.px = np.array([x.data_ptr() for x in self.X_c], dtype=np.uint64)
        self.pp = np.array([p.data_ptr() for p in self.piv], dtype=np.uint64)
        self.iter = np.zeros(count, dtype=np.int32)
        self.flags = np.zeros(count, dtype=np.uint32)
        self.info = np.zeros(count, dtype=np.int32)
        self.opts = default_opts(prec=prec, itermax=itermax, tol=tol,
                                 allow_fallback=int(bool(allow_fallback)))
        need = self.lib.mp_gesv_batched_workspace_bytes(count, self.n.ctypes.data, self.nrhs.ctypes.data,
                                                        ctypes.byref(self.opts))
        self.work = workspace(need, self.A_c[0].device if count else None)

    def run(self, stream=None):
        ret = self.lib.mp_gesv_batched(
            self.count, self.n.ctypes.data, self.nrhs.ctypes.data, self.pa.ctypes.data, self.lda.ctypes.data,
            self.pb.ctypes.data, self.ldb.ctypes.data, self.px.ctypes.data, self.ldx.ctypes.data,
            self.pp.ctypes.data, self.iter.ctypes.data, self.flags.ctypes.data, self.info.ctypes.data,
            self.work.data_ptr(), self.work.numel(), ctypes.byref(self.opts), _stream_ptr(stream))
        _check(ret, "mp_gesv_batched")
        return self

    def results(self):
        Xs = [x[:, 0] if v else x for x, v in zip(self.X_c, self.vec)]
        return Xs, [p[:int(m)] for p, m in zip(self.piv, self.n)], self.iter, self.flags, self.info


def gesv_batched(As, Bs, prec="fp32", itermax=30, tol=1e-14, allow_fallback=True, stream=None):
    """Solve the independent systems As[i] X_i = Bs[i] (n_i <= 512) in one
    persistent launch.  As, Bs: sequences of float64 CUDA tensors (B_i of
    shape (n_i,) or (n_i, nrhs_i)).  Returns (Xs, ipivs, iter, flags, info)
    with iter/flags/info numpy arrays."""
    plan = BatchedPlan(As, Bs, prec=prec, itermax=itermax, tol=tol, allow_fallback=allow_fallback)
    return plan.run(stream).results()


def gesv_host(A, B, prec="fp32", refine="classical", itermax=30, tol=1e-14, allow_fallback=True,
              nb_outer=0, work=None, stream=None):
    """Same as gesv with host (numpy, column-major float64) A and B; the host to
    device copies happen inside the C call."""
    import numpy as np
    lib = load()
    A = np.asfortranarray(A, dtype=np.float64)
    squeeze = np.asarray(B).ndim == 1
    B = np.asfortranarray(np.asarray(B, dtype=np.float64).reshape(A.shape[0], -1))
    n, nrhs = B.shape
    X = np.zeros((n, nrhs), dtype=np.float64, order="F")
    ipiv = np.zeros(max(n, 1), dtype=np.int32)
    opts = default_opts(prec=prec, refine=refine, itermax=itermax, tol=tol,
                        allow_fallback=int(bool(allow_fallback)), nb_outer=nb_outer)
    need = lib.mp_gesv_host_workspace_bytes(n, nrhs, ctypes.byref(opts))
    if work is None or work.numel() < need:
        work = workspace(need)
    st = mp_stats()
    ret = lib.mp_gesv_host(n, nrhs, A.ctypes.data, n, B.ctypes.data, n, X.ctypes.data, n,
                           ipiv.ctypes.data, work.data_ptr(), work.numel(), ctypes.byref(opts),
                           ctypes.byref(st), _stream_ptr(stream))
    _check(ret, "mp_gesv_host")
    return (X[:, 0] if squeeze else X), ipiv[:n], st.as_dict()


def factor_ld(n: int) -> int:
    return load().mp_factor_ld(n)


def convert(A, work=None, stream=None):
    """W = fl32(A) (row-major, ld = factor_ld(n)) and ||A||_inf.  Returns (W, anorm, flags)."""
    torch = _torch()
    lib = load()
    A = colmajor(A)
    n = A.shape[0]
    ldw = lib.mp_factor_ld(n)
    W = torch.zeros((n, ldw), dtype=torch.float32, device=A.device)
    anorm = torch.zeros(1, dtype=torch.float64, device=A.device)
    flags = torch.zeros(1, dtype=torch.int32, device=A.device)
    need = lib.mp_getrs_workspace_bytes(n, 1)
    if work is None or work.numel() < need:
        work = workspace(need, A.device)
    _check(lib.mp_convert(n, A.data_ptr(), _ld(A), W.data_ptr(), ldw, anorm.data_ptr(),
                          flags.data_ptr(), work.data_ptr(), work.numel(), _stream_ptr(stream)),
           "mp_convert")
    return W, anorm, flags


def getrf_lowp(W, prec="fp32", nb_outer=0, work=None, stream=None):
    """In-place LU with partial pivoting of the row-major FP32 W (n x ldw).
    Returns (ipiv, info, flags)."""
    torch = _torch()
    lib = load()
    n, ldw = W.shape
    opts = default_opts(prec=prec, nb_outer=nb_outer)
    ipiv = torch.zeros(max(n, 1), dtype=torch.int32, device=W.device)
    need = lib.mp_getrf_workspace_bytes(n, ctypes.byref(opts))
    if work is None or work.numel() < need:
        work = workspace(need, W.device)
    info = ctypes.c_int(0)
    flags = ctypes.c_uint32(0)
    _check(lib.mp_getrf_lowp(n, W.data_ptr(), ldw, ipiv.data_ptr(), ctypes.byref(opts),
                             work.data_ptr(), work.numel(), ctypes.byref(info), ctypes.byref(flags),
                             _stream_ptr(stream)), "mp_getrf_lowp")
    return ipiv[:n], info.value, flags.value


def potrf_lowp(W, prec="fp32", nb_outer=0, work=None, stream=None):
    """In-place Cholesky (lower) of the row-major FP32 W (n x ldw).
    Returns (info, flags)."""
    lib = load()
    n, ldw = W.shape
    opts = default_opts(prec=prec, nb_outer=nb_outer)
    need = lib.mp_getrf_workspace_bytes(n, ctypes.byref(opts))
    if work is None or work.numel() < need:
        work = workspace(need, W.device)
    info = ctypes.c_int(0)
    flags = ctypes.c_uint32(0)
    _check(lib.mp_potrf_lowp(n, W.data_ptr(), ldw, ctypes.byref(opts), work.data_ptr(), work.numel(),
                             ctypes.byref(info), ctypes.byref(flags), _stream_ptr(stream)),
           "mp_potrf_lowp")
    return info.value, flags.value


def getrs_lowp(W, ipiv, R, work=None, stream=None):
    """z = U^{-1} L^{-1} P r with the FP32 factors (scaled by a power of two); FP64 in/out."""
    torch = _torch()
    lib = load()
    n, ldw = W.shape
    squeeze = R.dim() == 1
    R = colmajor(R)
    nrhs = R.shape[1]
    Z = torch.empty((nrhs, n), dtype=torch.float64, device=W.device).t()
    need = lib.mp_getrs_workspace_bytes(n, nrhs)
    if work is None or work.numel() < need:
        work = workspace(need, W.device)
    _check(lib.mp_getrs_lowp(n, nrhs, W.data_ptr(), ldw, ipiv.data_ptr(), R.data_ptr(), _ld(R),
                             Z.data_ptr(), _ld(Z), work.data_ptr(), work.numel(),
                             _stream_ptr(stream)), "mp_getrs_lowp")
    return Z[:, 0] if squeeze else Z


def residual(A, X, B, work=None, stream=None):
    """R = B - A X in FP64 (Algorithm 1 step 4)."""
    torch = _torch()
    lib = load()
    A = colmajor(A)
    squeeze = X.dim() == 1
    X = colmajor(X)
    B = colmajor(B)
    n, nrhs = X.shape
    R = torch.empty((nrhs, n), dtype=torch.float64, device=A.device).t()
    need = lib.mp_residual_workspace_bytes(n, nrhs)
    if work is None or work.numel() < need:
        work = workspace(need, A.device)
    _check(lib.mp_residual(n, nrhs, A.data_ptr(), _ld(A), X.data_ptr(), _ld(X),
                           B.data_ptr(), _ld(B), R.data_ptr(), _ld(R), work.data_ptr(),
                           work.numel(), _stream_ptr(stream)), "mp_residual")
    return R[:, 0] if squeeze else R


def lowp_gemm_update(C, L, U, prec="bf16", work=None, stream=None):
    """C -= fl_p(L) fl_p(U) in place; C, L, U row-major (contiguous) FP32 CUDA tensors."""
    lib = load()
    M, K = L.shape
    K2, N = U.shape
    assert K == K2 and tuple(C.shape) == (M, N)
    p = PREC[prec] if isinstance(prec, str) else int(prec)
    need = lib.mp_lowp_gemm_workspace_bytes(M, N, K, p)
    if work is None or work.numel() < need:
        work = workspace(need, C.device)
    _check(lib.mp_lowp_gemm_update(p, M, N, K, L.data_ptr(), L.stride(0), U.data_ptr(), U.stride(0),
                                   C.data_ptr(), C.stride(0), work.data_ptr(), work.numel(),
                                   _stream_ptr(stream)), "mp_lowp_gemm_update")
    return C


def selftest_wait_timeout(site: int, limit_ns: int, stream=None):
    """Runs one of the library's bounded device waits on a condition nothing
    satisfies (site 2: triangular-solve grid barrier, 3: panel mbarrier wait,
    4: tensor-core mbarrier wait) with the given limit.  Returns (flags,
    recorded site, CTAs past the barrier)."""
    lib = load()
    work = workspace(lib.mp_selftest_workspace_bytes())
    fl, si, pa = ctypes.c_uint(0), ctypes.c_int(0), ctypes.c_int(0)
    _check(lib.mp_selftest_wait_timeout(int(site), int(limit_ns), work.data_ptr(), work.numel(), ctypes.byref(fl),
                                        ctypes.byref(si), ctypes.byref(pa), _stream_ptr(stream)),
           "mp_selftest_wait_timeout")
    return fl.value, si.value, pa.value


def shard_by_cost(ns, world: int):
    """Partition of a batch of systems over `world` ranks by cost n^3 (the
    O(n^3) factorization dominates): systems in decreasing n^3 (ties: lower
    index first) each go to the rank with the least cost so far (ties: lower
    rank).  Returns one list of system indices per rank, in the order the
    systems were assigned (longest first)."""
    order = sorted(range(len(ns)), key=lambda i: (-int(ns[i]) ** 3, i))
    load = [0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += int(ns[i]) ** 3
    return parts


def gesv_batched_sharded(ns, get_system, group=None, solve=None, **kw):
    """A batch of independent systems spread over the ranks of a
    torch.distributed group by cost (shard_by_cost), each rank solving its
    share in one mp_gesv_batched launch; there is no exchange on the data
    path.  ns: every system's order (the same list on every rank);
    get_system(i) -> (A_i, B_i) device tensors of system i, called only for
    this rank's systems; solve(As, Bs) -> (Xs, iter, flags) defaults to
    gesv_batched with **kw.  Afterwards one all-gather gives every rank the
    iteration counts and flags of the whole batch.  Returns (mine, Xs, iter,
    flags): this rank's system indices and solutions, and the batch's
    iter/flags as numpy arrays indexed by system."""
    import numpy as np
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    mine = shard_by_cost(ns, world)[rank]
    if solve is None:
        def solve(As, Bs):
            Xs, _, it, fl, _ = gesv_batched(As, Bs, **kw)
            return Xs, it, fl
    if mine:
        systems = [get_system(i) for i in mine]
        Xs, it, fl = solve([a for a, _ in systems], [b for _, b in systems])
    else:
        Xs, it, fl = [], np.zeros(0, dtype=np.int32), np.zeros(0, dtype=np.uint32)
    local = (list(mine), [int(v) for v in it], [int(v) for v in fl])
    gathered = [None] * world
    dist.all_gather_object(gathered, local, group=group)
    iters = np.full(len(ns), np.iinfo(np.int32).min, dtype=np.int64)
    flags = np.zeros(len(ns), dtype=np.uint64)
    for idx, its, fls in gathered:
        iters[idx] = its
        flags[idx] = fls
    return mine, Xs, iters, flags


def batched_schedule():
    """The batched solver's active tile schedule: list of (nmax, panel width)."""
    import numpy as np
    lib = load()
    cnt = ctypes.c_int(0)
    nm = np.zeros(64, dtype=np.int32)
    nb = np.zeros(64, dtype=np.int32)
    _check(lib.mp_batched_get_schedule(64, ctypes.byref(cnt), nm.ctypes.data, nb.ctypes.data),
           "mp_batched_get_schedule")
    return [(int(nm[i]), int(nb[i])) for i in range(cnt.value)]


def set_batched_schedule(entries=None):
    """Replaces the batched solver's tile schedule for this process with
    entries [(nmax, panel width), ...]; None restores the built-in table."""
    import numpy as np
    lib = load()
    if not entries:
        _check(lib.mp_batched_set_schedule(0, None, None), "mp_batched_set_schedule")
        return
    nm = np.array([e[0] for e in entries], dtype=np.int32)
    nb = np.array([e[1] for e in entries], dtype=np.int32)
    _check(lib.mp_batched_set_schedule(len(entries), nm.ctypes.data, nb.ctypes.data), "mp_batched_set_schedule")


def gesv_dd(A, B, itermax=10, work=None, stream=None):
    """Solve A X = B to double-double accuracy (Section 5's extra-precise
    refinement with FP64 factors).  A: (n, n) float64 CUDA tensor, B: (n,) or
    (n, nrhs).  Returns (Xhi, Xlo, ipiv, stats) with X = Xhi + Xlo."""
    torch = _torch()
    lib = load()
    A = colmajor(A)
    squeeze = B.dim() == 1
    B = colmajor(B)
    n, nrhs = B.shape
    Xhi = torch.empty((nrhs, n), dtype=torch.float64, device=A.device).t()
    Xlo = torch.empty((nrhs, n), dtype=torch.float64, device=A.device).t()
    ipiv = torch.empty(max(n, 1), dtype=torch.int32, device=A.device)
    need = lib.mp_gesv_dd_workspace_bytes(n, nrhs)
    if work is None or work.numel() < need:
        work = workspace(need, A.device)
    st = mp_stats()
    ret = lib.mp_gesv_dd(n, nrhs, A.data_ptr(), _ld(A), B.data_ptr(), _ld(B), Xhi.data_ptr(), Xlo.data_ptr(),
                         _ld(Xhi), ipiv.data_ptr(), int(itermax), work.data_ptr(), work.numel(), ctypes.byref(st),
                         _stream_ptr(stream))
    _check(ret, "mp_gesv_dd")
    d = st.as_dict()
    d["info_fp64"] = ret
    if squeeze:
        return Xhi[:, 0], Xlo[:, 0], ipiv[:n], d
    return Xhi, Xlo, ipiv[:n], d


def gels(A, B, prec="fp32", refine="classical", alpha=0.0, allow_fallback=True, work=None, stream=None):
    """Least squares min ||B - A X||_2 (A: (m, n) float64 CUDA tensor, m >= n,
    full column rank; B: (m,) or (m, nrhs)) by refinement of the augmented
    system.  Returns (X, R, stats) with R = B - A X."""
    torch = _torch()
    lib = load()
    A = colmajor(A)
    squeeze = B.dim() == 1
    B = colmajor(B)
    m, n = A.shape
    nrhs = B.shape[1]
    opts = default_opts(prec=prec, refine=refine, allow_fallback=int(bool(allow_fallback)))
    X = torch.empty((nrhs, n), dtype=torch.float64, device=A.device).t()
    R = torch.empty((nrhs, m), dtype=torch.float64, device=A.device).t()
    need = lib.mp_gels_workspace_bytes(m, n, nrhs, ctypes.byref(opts))
    if work is None or work.numel() < need:
        work = workspace(need, A.device)
    st = mp_stats()
    ret = lib.mp_gels(m, n, nrhs, A.data_ptr(), _ld(A), B.data_ptr(), _ld(B), X.data_ptr(), _ld(X), R.data_ptr(),
                      _ld(R), float(alpha), work.data_ptr(), work.numel(), ctypes.byref(opts), ctypes.byref(st),
                      _stream_ptr(stream))
    _check(ret, "mp_gels")
    d = st.as_dict()
    d["info_fp64"] = ret
    if squeeze:
        return X[:, 0], R[:, 0], d
    return X, R, d


# ---------------------------------------------------------------------------
# Sparse systems: Algorithm 2 (Section 2.2), FGMRES(m_out)-GMRES_SP(m_in)
# ---------------------------------------------------------------------------
def sparse_opts(m_out=20, m_in=30, inner="fp32", max_cycles=100, tol=1e-14) -> mp_sparse_opts:
    o = mp_sparse_opts()
    load().mp_sparse_default_opts(ctypes.byref(o))
    o.m_out, o.m_in, o.max_cycles, o.tol = int(m_out), int(m_in), int(max_cycles), float(tol)
    o.inner = INNER[inner] if isinstance(inner, str) else int(inner)
    return o


def _csr_args(indptr, indices, values):
    torch = _torch()
    for t, dt, name in ((indptr, torch.int32, "indptr"), (indices, torch.int32, "indices"),
                        (values, torch.float64, "values")):
        if not t.is_cuda or t.dtype != dt or not t.is_contiguous():
            raise MpError(f"{name} must be a contiguous CUDA tensor of {dt}")
    return indptr.numel() - 1, values.numel()


def fgmres(indptr, indices, values, b, m_out=20, m_in=30, inner="fp32", max_cycles=100, tol=1e-14,
           work=None, stream=None):
    """Solve A x = b for a CSR matrix (int32 indptr/indices, float64 values,
    CUDA tensors) by FGMRES(m_out) preconditioned by one cycle of GMRES(m_in)
    in FP32 (inner="fp32"), FP64 ("fp64") or without a preconditioner
    ("none": plain restarted GMRES(m_out)).  Returns (x, stats)."""
    torch = _torch()
    lib = load()
    n, nnz = _csr_args(indptr, indices, values)
    b = b.contiguous()
    x = torch.empty(n, dtype=torch.float64, device=b.device)
    o = sparse_opts(m_out, m_in, inner, max_cycles, tol)
    need = lib.mp_fgmres_workspace_bytes(n, nnz, ctypes.byref(o))
    if work is None or work.numel() < need:
        work = workspace(need, b.device)
    st = mp_sparse_stats()
    ret = lib.mp_fgmres(n, nnz, indptr.data_ptr(), indices.data_ptr(), values.data_ptr(), b.data_ptr(),
                        x.data_ptr(), work.data_ptr(), work.numel(), ctypes.byref(o), ctypes.byref(st),
                        _stream_ptr(stream))
    _check(ret, "mp_fgmres")
    return x, st.as_dict()


def sparse_gmres_cycle(indptr, indices, values, v, m, inner="fp32", work=None, stream=None):
    """One cycle of GMRES(m) for A z = v from z = 0 in FP32 or FP64 (the inner
    solver of Algorithm 2).  Returns (z, steps)."""
    torch = _torch()
    lib = load()
    n, nnz = _csr_args(indptr, indices, values)
    v = v.contiguous()
    z = torch.empty(n, dtype=torch.float64, device=v.device)
    o = sparse_opts(1, m, inner)
    need = lib.mp_fgmres_workspace_bytes(n, nnz, ctypes.byref(o))
    if work is None or work.numel() < need:
        work = workspace(need, v.device)
    steps = ctypes.c_int(0)
    ret = lib.mp_sparse_gmres_cycle(n, nnz, indptr.data_ptr(), indices.data_ptr(), values.data_ptr(), v.data_ptr(),
                                    z.data_ptr(), int(m), INNER[inner], work.data_ptr(), work.numel(),
                                    ctypes.byref(steps), _stream_ptr(stream))
    _check(ret, "mp_sparse_gmres_cycle")
    return z, steps.value


def csr_spmv(indptr, indices, values, x, prec="fp64", stream=None):
    """y = A x for a CSR matrix, in FP64 or FP32 (values and x rounded)."""
    torch = _torch()
    lib = load()
    n, nnz = _csr_args(indptr, indices, values)
    x = x.contiguous()
    y = torch.empty(n, dtype=torch.float64, device=x.device)
    ret = lib.mp_csr_spmv(n, nnz, indptr.data_ptr(), indices.data_ptr(), values.data_ptr(), x.data_ptr(),
                          y.data_ptr(), PREC[prec], _stream_ptr(stream))
    _check(ret, "mp_csr_spmv")
    return y
