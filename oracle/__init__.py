"""CPU oracle for the mixed-precision iterative-refinement solver.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / reference leg may import this package.  It shares
no code with the CUDA library (``paper_0808_2794_gb300``), and the CUDA library
never imports it.

The arithmetic lives in ``oracle.c`` (plain C, FP64 unless the routine is the
paper's single-precision factorization).  ``exact.py`` holds exact rational
(``fractions.Fraction``) versions used to pin the C code.  This module only
compiles ``oracle.c`` with gcc and marshals numpy arrays (column-major).

Citations refer to Baboulin et al., "Accelerating Scientific Computations with
Mixed Precision Algorithms": Algorithm 1 (Section 2.1), Eq. (2) and
Algorithm 2 (Section 2.2), the accuracy test (Section 3), the LAPACK mapping
(Section 3.1.1), the convergence condition and iteration-count formula
(Section 4).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

FALLBACK = 1
STALLED = 2
BREAKDOWN = 4
NONFINITE = 8


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (gcc, OpenMP, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            I = ctypes.c_int
            D = ctypes.c_double
            sig = {
                "or_set_threads": (I, [I]),
                "or_dgetrf": (I, [I, P, I, P]),
                "or_sgetrf": (I, [I, P, I, P]),
                "or_dgetrs": (None, [I, I, P, I, P, P, I]),
                "or_sgetrs": (None, [I, I, P, I, P, P, I]),
                "or_dgetrs_trans": (None, [I, I, P, I, P, P, I]),
                "or_dpotrf": (I, [I, P, I]),
                "or_spotrf": (I, [I, P, I]),
                "or_dpotrs": (None, [I, I, P, I, P, I]),
                "or_spotrs": (None, [I, I, P, I, P, I]),
                "or_dresidual": (None, [I, I, P, I, P, I, P, I, P, I]),
                "or_dresidual_dot2": (None, [I, I, P, I, P, I, P, I, P, I]),
                "or_dmatvec_dot2": (None, [I, I, P, I, P, I, P, I]),
                "or_dnorm_inf": (D, [I, I, P, I]),
                "or_bwd_err": (None, [I, I, P, I, P, I, P, I, P]),
                "or_gesv_ir": (I, [I, I, P, I, P, I, P, I, I, I, D, D, I, P, P, P, P, P]),
                "or_posv_ir": (I, [I, I, P, I, P, I, P, I, I, I, D, D, I, P, P, P]),
                "or_gesv_dd": (I, [I, I, P, I, P, I, P, P, I, I, P]),
                "or_kappa_inf": (D, [I, P, I]),
                "or_kappa_1_est": (D, [I, P, I]),
                "or_dinvnorm1_est_lu": (D, [I, P, I, P, I]),
                "or_round_bf16": (D, [D]),
                "or_round_fp16": (D, [D]),
                "or_round_e4m3": (D, [D]),
                "or_gmres_ir": (I, [I, P, I, P, P, I, I, D, D, P, P]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _f(a, dtype):
    """Column-major contiguous copy (or view) of a 1-D/2-D array."""
    a = np.asarray(a, dtype=dtype)
    if a.ndim == 1:
        a = a.reshape(-1, 1)
    return np.asfortranarray(a)


def _p(a):
    return ctypes.c_void_p(a.ctypes.data)


def set_threads(nt: int = 0) -> int:
    """Set the OpenMP thread count (0 keeps it); returns the count in use."""
    return _load().or_set_threads(int(nt))


def getrf(A, prec: int = 64):
    """PA = LU with partial pivoting (Section 2.1; Algorithm 1 step 1).

    Returns (LU, ipiv, info); ipiv is 1-based LAPACK style.
    """
    lib = _load()
    dt = np.float64 if prec == 64 else np.float32
    F = _f(A, dt).copy(order="F")
    n = F.shape[0]
    ipiv = np.zeros(max(n, 1), dtype=np.int32)
    fn = lib.or_dgetrf if prec == 64 else lib.or_sgetrf
    info = fn(n, _p(F), max(n, 1), _p(ipiv))
    return F, ipiv[:n], info


def getrs(LU, ipiv, B, prec: int = 64):
    """Solve with LU factors: Ly = Pb, Ux = y (Algorithm 1 steps 2-3, 5-6)."""
    lib = _load()
    dt = np.float64 if prec == 64 else np.float32
    F = _f(LU, dt)
    squeeze = np.asarray(B).ndim == 1
    X = _f(B, dt).copy(order="F")
    n, nrhs = X.shape
    piv = np.ascontiguousarray(ipiv, dtype=np.int32)
    fn = lib.or_dgetrs if prec == 64 else lib.or_sgetrs
    fn(n, nrhs, _p(F), max(n, 1), _p(piv), _p(X), max(n, 1))
    return X[:, 0] if squeeze else X


def getrs_trans(LU, ipiv, B):
    """Solve A^T x = b with the FP64 LU factors of A."""
    lib = _load()
    F = _f(LU, np.float64)
    squeeze = np.asarray(B).ndim == 1
    X = _f(B, np.float64).copy(order="F")
    n, nrhs = X.shape
    piv = np.ascontiguousarray(ipiv, dtype=np.int32)
    lib.or_dgetrs_trans(n, nrhs, _p(F), max(n, 1), _p(piv), _p(X), max(n, 1))
    return X[:, 0] if squeeze else X


def potrf(A, prec: int = 64):
    """Lower Cholesky A = L L^T (SPOTRF/DPOTRF, Section 3.1.1).  Returns (L, info);
    the strict upper triangle of the returned array is the untouched input."""
    lib = _load()
    dt = np.float64 if prec == 64 else np.float32
    F = _f(A, dt).copy(order="F")
    n = F.shape[0]
    fn = lib.or_dpotrf if prec == 64 else lib.or_spotrf
    info = fn(n, _p(F), max(n, 1))
    return F, info


def potrs(L, B, prec: int = 64):
    lib = _load()
    dt = np.float64 if prec == 64 else np.float32
    F = _f(L, dt)
    squeeze = np.asarray(B).ndim == 1
    X = _f(B, dt).copy(order="F")
    n, nrhs = X.shape
    fn = lib.or_dpotrs if prec == 64 else lib.or_spotrs
    fn(n, nrhs, _p(F), max(n, 1), _p(X), max(n, 1))
    return X[:, 0] if squeeze else X


def residual(A, X, B, compensated: bool = False):
    """R = B - A X in FP64 (Algorithm 1 step 4); compensated=True uses Dot2."""
    lib = _load()
    Af = _f(A, np.float64)
    squeeze = np.asarray(X).ndim == 1
    Xf = _f(X, np.float64)
    Bf = _f(B, np.float64)
    n, nrhs = Xf.shape
    R = np.zeros((n, nrhs), dtype=np.float64, order="F")
    fn = lib.or_dresidual_dot2 if compensated else lib.or_dresidual
    fn(n, nrhs, _p(Af), max(n, 1), _p(Xf), max(n, 1), _p(Bf), max(n, 1), _p(R), max(n, 1))
    return R[:, 0] if squeeze else R


def matvec_dot2(A, X):
    """B = A X with the compensated Dot2 product (right-hand-side construction)."""
    lib = _load()
    Af = _f(A, np.float64)
    squeeze = np.asarray(X).ndim == 1
    Xf = _f(X, np.float64)
    n, nrhs = Xf.shape
    B = np.zeros((n, nrhs), dtype=np.float64, order="F")
    lib.or_dmatvec_dot2(n, nrhs, _p(Af), max(n, 1), _p(Xf), max(n, 1), _p(B), max(n, 1))
    return B[:, 0] if squeeze else B


def norm_inf(A) -> float:
    lib = _load()
    Af = _f(A, np.float64)
    m, n = Af.shape
    return float(lib.or_dnorm_inf(m, n, _p(Af), max(m, 1)))


def bwd_err(A, X, B):
    """Per-column ||b - Ax||_inf / (||A||_inf ||x||_inf + ||b||_inf), compensated residual."""
    lib = _load()
    Af = _f(A, np.float64)
    Xf = _f(X, np.float64)
    Bf = _f(B, np.float64)
    n, nrhs = Xf.shape
    out = np.zeros(max(nrhs, 1), dtype=np.float64)
    lib.or_bwd_err(n, nrhs, _p(Af), max(n, 1), _p(Xf), max(n, 1), _p(Bf), max(n, 1), _p(out))
    return out[:nrhs]


def gesv_ir(A, B, factor_prec: int = 32, itermax: int = 30, tol: float = 1e-14,
            stall_ratio: float = 0.5, allow_fallback: bool = True):
    """Algorithm 1: mixed-precision iterative refinement (Section 2.1).

    Returns dict(X, info, iter, flags, bwd, hist).
    """
    lib = _load()
    Af = _f(A, np.float64)
    squeeze = np.asarray(B).ndim == 1
    Bf = _f(B, np.float64)
    n, nrhs = Bf.shape
    X = np.zeros((n, nrhs), dtype=np.float64, order="F")
    it = ctypes.c_int(0)
    fl = ctypes.c_uint(0)
    bw = ctypes.c_double(0)
    nh = ctypes.c_int(0)
    hist = np.zeros(32, dtype=np.float64)
    info = lib.or_gesv_ir(n, nrhs, _p(Af), max(n, 1), _p(Bf), max(n, 1), _p(X), max(n, 1),
                          int(factor_prec), int(itermax), float(tol), float(stall_ratio),
                          int(bool(allow_fallback)), ctypes.byref(it), ctypes.byref(fl),
                          ctypes.byref(bw), ctypes.byref(nh), _p(hist))
    return dict(X=X[:, 0] if squeeze else X, info=info, iter=it.value, flags=fl.value,
                bwd=bw.value, hist=hist[:nh.value].copy())


def gesv_dd(A, B, itermax: int = 10):
    """Section 5's extra-precise refinement with FP64 factors: returns
    dict(Xhi, Xlo, info, iter) with X = Xhi + Xlo in double-double."""
    lib = _load()
    Af = _f(A, np.float64)
    squeeze = np.asarray(B).ndim == 1
    Bf = _f(B, np.float64)
    n, nrhs = Bf.shape
    Xh = np.zeros((n, nrhs), dtype=np.float64, order="F")
    Xl = np.zeros((n, nrhs), dtype=np.float64, order="F")
    it = ctypes.c_int(0)
    info = lib.or_gesv_dd(n, nrhs, _p(Af), max(n, 1), _p(Bf), max(n, 1), _p(Xh), _p(Xl), max(n, 1),
                          int(itermax), ctypes.byref(it))
    if squeeze:
        Xh, Xl = Xh[:, 0], Xl[:, 0]
    return dict(Xhi=Xh, Xlo=Xl, info=info, iter=it.value)


def gels_aug(A, B, alpha: float = 0.0):
    """Least squares min ||b - A x||_2 (Section 6's extension) through the
    augmented system [alpha I, A; A^T, 0] [r / alpha; x] = [b; 0], solved by
    the oracle's Algorithm 1 with FP64 factors; alpha = 0 picks the power of
    two nearest ||A||_F / sqrt(8 n).  Returns dict(X, R, alpha, info)."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    Bm = np.asarray(B, dtype=np.float64).reshape(m, -1)
    if alpha == 0.0:
        t = float(np.sqrt(np.sum(A * A) / (8.0 * n)))
        alpha = 2.0 ** int(round(np.log2(t))) if t > 0 else 1.0
    K = np.zeros((m + n, m + n))
    K[:m, :m] = alpha * np.eye(m)
    K[:m, m:] = A
    K[m:, :m] = A.T
    F = np.zeros((m + n, Bm.shape[1]))
    F[:m] = Bm
    r = gesv_ir(np.asfortranarray(K), np.asfortranarray(F), factor_prec=64)
    Y = r["X"].reshape(m + n, -1)
    return dict(X=Y[m:], R=alpha * Y[:m], alpha=alpha, info=r["info"])


def posv_ir(A, B, factor_prec: int = 32, itermax: int = 30, tol: float = 1e-14,
            stall_ratio: float = 0.5, allow_fallback: bool = True):
    """Algorithm 1 with a Cholesky factorization (Section 3.1.1, Section 6)."""
    lib = _load()
    Af = _f(A, np.float64)
    squeeze = np.asarray(B).ndim == 1
    Bf = _f(B, np.float64)
    n, nrhs = Bf.shape
    X = np.zeros((n, nrhs), dtype=np.float64, order="F")
    it = ctypes.c_int(0)
    fl = ctypes.c_uint(0)
    bw = ctypes.c_double(0)
    info = lib.or_posv_ir(n, nrhs, _p(Af), max(n, 1), _p(Bf), max(n, 1), _p(X), max(n, 1),
                          int(factor_prec), int(itermax), float(tol), float(stall_ratio),
                          int(bool(allow_fallback)), ctypes.byref(it), ctypes.byref(fl),
                          ctypes.byref(bw))
    return dict(X=X[:, 0] if squeeze else X, info=info, iter=it.value, flags=fl.value,
                bwd=bw.value)


def gmres_ir(A, b, restart: int = 30, outer_max: int = 30, tol: float = 1e-14,
             inner_tol: float = 1e-6):
    """GMRES-based refinement preconditioned by the FP32 LU (Section 2.2).

    Returns dict(x, outer, nmatvec, bwd); outer = -1 if the FP32 factorization broke down.
    """
    lib = _load()
    Af = _f(A, np.float64)
    bf = np.ascontiguousarray(b, dtype=np.float64).reshape(-1)
    n = bf.shape[0]
    x = np.zeros(n, dtype=np.float64)
    nmv = ctypes.c_int(0)
    bw = ctypes.c_double(0)
    outer = lib.or_gmres_ir(n, _p(Af), max(n, 1), _p(bf), _p(x), int(restart), int(outer_max),
                            float(tol), float(inner_tol), ctypes.byref(nmv), ctypes.byref(bw))
    return dict(x=x, outer=outer, nmatvec=nmv.value, bwd=bw.value)


def kappa_inf(A) -> float:
    """Exact kappa_inf from an explicit FP64 inverse (n solves)."""
    lib = _load()
    Af = _f(A, np.float64)
    return float(lib.or_kappa_inf(Af.shape[0], _p(Af), max(Af.shape[0], 1)))


def kappa_inf_est_lu(A, LU, ipiv) -> float:
    """kappa_inf(A) estimate ||A||_inf * est(||A^{-1}||_inf) from existing FP64
    LU factors of A (Hager-Higham on A^{-T}; a lower bound)."""
    lib = _load()
    F = _f(LU, np.float64)
    piv = np.ascontiguousarray(ipiv, dtype=np.int32)
    n = F.shape[0]
    return norm_inf(A) * float(lib.or_dinvnorm1_est_lu(n, _p(F), max(n, 1), _p(piv), 1))


def kappa_1_est(A) -> float:
    """Hager-Higham 1-norm condition estimate (DGECON's algorithm, Table 7)."""
    lib = _load()
    Af = _f(A, np.float64)
    return float(lib.or_kappa_1_est(Af.shape[0], _p(Af), max(Af.shape[0], 1)))


def round_to(x, prec: str):
    """Round each element to bf16 / fp16 / e4m3 (RNE; e4m3 saturating)."""
    lib = _load()
    fn = {"bf16": lib.or_round_bf16, "fp16": lib.or_round_fp16, "e4m3": lib.or_round_e4m3}[prec]
    arr = np.asarray(x, dtype=np.float64)
    out = np.array([fn(float(v)) for v in arr.reshape(-1)], dtype=np.float64)
    return out.reshape(arr.shape)
