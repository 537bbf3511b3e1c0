"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the solver: it only draws random numbers
(numpy PCG64 via ``default_rng(seed)``) and assembles the systems to be solved.
Both the CUDA path's tests/benchmark and the CPU oracle's tests take their
inputs from here.

The paper evaluates dense random systems (Table 3, Section 3.1.1), matrices of
prescribed condition number (200 random 200x200 matrices per kappa, Section 4,
Fig. 4 protocol) and uniform-random matrices (Section 5).  All matrices are
returned column-major (``numpy`` Fortran order); column j of A is the j-th
consecutive block of n draws.  Per seed the draw order is A, then X_true (or
B), then any further array.  Right-hand sides are B = A @ X_true formed once
in FP64 by numpy; every consumer uses that same array.
"""
from __future__ import annotations

import math

import numpy as np


def _colmajor_normal(rng, n, m=None):
    m = n if m is None else m
    # draw G with shape (m, n) row-major and view its transpose: column j of the
    # result is the j-th block of n consecutive draws; no copy is made.
    return rng.standard_normal((m, n)).T


def dense_system(n: int, nrhs: int = 1, seed: int = 0):
    """A ~ N(0,1) i.i.d., X_true ~ U[-1,1], B = A X_true (dense LU workloads)."""
    rng = np.random.default_rng(seed)
    A = _colmajor_normal(rng, n)
    X = np.asfortranarray(rng.uniform(-1.0, 1.0, size=(nrhs, n)).T)
    B = np.asfortranarray(A @ X)
    return A, B, X


def haar_orthogonal(rng, n):
    """Q of the QR of a Gaussian matrix with the signs of diag(R) folded in
    (Haar-distributed orthogonal matrix, Mezzadri 2007)."""
    G = rng.standard_normal((n, n))
    Q, R = np.linalg.qr(G)
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return Q * d[None, :]


def conditioned_system(n: int, kappa: float, nrhs: int = 1, spd: bool = False, seed: int = 0):
    """A = U diag(s) V^T (general) or U diag(s) U^T (SPD, symmetrized as
    (A + A^T)/2) with Haar U, V and s_i = kappa^{-i/(n-1)}, i = 0..n-1, so the
    2-norm condition number is kappa.  X_true ~ U[-1,1], B = A X_true."""
    rng = np.random.default_rng(seed)
    U = haar_orthogonal(rng, n)
    V = U if spd else haar_orthogonal(rng, n)
    i = np.arange(n, dtype=np.float64)
    s = kappa ** (-i / max(n - 1, 1))
    A = (U * s[None, :]) @ V.T
    if spd:
        A = 0.5 * (A + A.T)
    A = np.asfortranarray(A)
    X = np.asfortranarray(rng.uniform(-1.0, 1.0, size=(nrhs, n)).T)
    B = np.asfortranarray(A @ X)
    return A, B, X


def conditioned_family(n: int, kappas, nrhs: int = 1, spd: bool = False, seed: int = 0):
    """The systems conditioned_system(n, kappa, nrhs, spd, seed) for every
    kappa in kappas, with the Haar factors and X_true drawn once: per seed the
    draws do not depend on kappa, so each (A, B, X) equals the one that
    conditioned_system returns.  Yields (kappa, A, B, X)."""
    rng = np.random.default_rng(seed)
    U = haar_orthogonal(rng, n)
    V = U if spd else haar_orthogonal(rng, n)
    X = np.asfortranarray(rng.uniform(-1.0, 1.0, size=(nrhs, n)).T)
    i = np.arange(n, dtype=np.float64)
    for kappa in kappas:
        s = kappa ** (-i / max(n - 1, 1))
        A = (U * s[None, :]) @ V.T
        if spd:
            A = 0.5 * (A + A.T)
        A = np.asfortranarray(A)
        yield kappa, A, np.asfortranarray(A @ X), X


def conditioned_batch_family(n: int, count: int, kappas, seed: int = 0):
    """The Fig. 4 protocol (Section 4): for every kappa in kappas, `count`
    random n x n general systems of 2-norm condition number kappa,
    A_i = U_i diag(s) V_i^T with Haar U_i, V_i and s_j = kappa^{-j/(n-1)},
    X_true ~ U[-1,1], b = A x_true (nrhs = 1).  The pairs (U_i, V_i) and
    x_true,i are drawn once (in the order U_1, V_1, x_1, U_2, ...) and reused
    for every kappa.  Yields (kappa, As, Bs, Xs) with lists of length count."""
    rng = np.random.default_rng(seed)
    pairs = []
    for _ in range(count):
        U = haar_orthogonal(rng, n)
        V = haar_orthogonal(rng, n)
        x = rng.uniform(-1.0, 1.0, size=(n, 1))
        pairs.append((U, V, np.asfortranarray(x)))
    i = np.arange(n, dtype=np.float64)
    for kappa in kappas:
        s = kappa ** (-i / max(n - 1, 1))
        As, Bs, Xs = [], [], []
        for U, V, x in pairs:
            A = np.asfortranarray((U * s[None, :]) @ V.T)
            As.append(A)
            Bs.append(np.asfortranarray(A @ x))
            Xs.append(x)
        yield kappa, As, Bs, Xs


def batched_systems(count: int = 4096, seed: int = 0, nmin: int = 16, nmax: int = 512,
                    max_nrhs: int = 4):
    """``count`` independent systems, n = round(exp(U[ln nmin, ln nmax])),
    nrhs ~ U{1..max_nrhs}, A = N(0,1) + n I (diagonally dominant), X_true ~
    U[-1,1], B = A X_true.  Returns lists (A_list, B_list, X_list)."""
    rng = np.random.default_rng(seed)
    ns = np.rint(np.exp(rng.uniform(math.log(nmin), math.log(nmax), size=count))).astype(int)
    nrhs = rng.integers(1, max_nrhs + 1, size=count)
    As, Bs, Xs = [], [], []
    for n, r in zip(ns, nrhs):
        A = _colmajor_normal(rng, int(n)).copy(order="F")
        A[np.diag_indices(int(n))] += float(n)
        X = np.asfortranarray(rng.uniform(-1.0, 1.0, size=(int(r), int(n))).T)
        As.append(A)
        Xs.append(X)
        Bs.append(np.asfortranarray(A @ X))
    return As, Bs, Xs


def adjoint_problem(n: int = 2048, nrhs: int = 8, seed: int = 0):
    """A = N(0,1) + sqrt(n) I, B ~ N(0,1), Wt ~ N(0,1) (loss = sum(Wt * X))."""
    rng = np.random.default_rng(seed)
    A = _colmajor_normal(rng, n).copy(order="F")
    A[np.diag_indices(n)] += math.sqrt(n)
    B = np.asfortranarray(rng.standard_normal((nrhs, n)).T)
    Wt = np.asfortranarray(rng.standard_normal((nrhs, n)).T)
    return A, B, Wt


def small_integer_matrix(n: int, seed: int = 0, lo: int = -9, hi: int = 9):
    """Random small-integer matrix (exactly representable in every precision
    used here) for exact rational pins."""
    rng = np.random.default_rng(seed)
    return np.asfortranarray(rng.integers(lo, hi + 1, size=(n, n)).astype(np.float64))
