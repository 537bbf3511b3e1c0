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


# ---------------------------------------------------------------------------
# Sparse systems for the inner-outer iterative method (Algorithm 2,
# Section 2.2).  The paper's Table 2 matrices come from a public collection
# that is not available here; these seeded matrices stand in for them with
# the same orders, nonzeros per row, symmetry and rough condition numbers.
# Returned as CSR arrays (indptr int32, indices int32 sorted within each row,
# data FP64), every row holding its diagonal entry.
# ---------------------------------------------------------------------------
def _csr_from_coo(n, rows, cols, vals):
    import scipy.sparse as sp
    A = sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()  # duplicates summed
    A.sort_indices()
    return (A.indptr.astype(np.int32), A.indices.astype(np.int32), A.data.astype(np.float64))


def sparse_stencil27(g: int, beta: float = 0.3, seed: int = 0):
    """Convection-diffusion on a g x g x g grid with the 27-point stencil
    (Dirichlet boundary; n = g^3, 27 entries in interior rows): diagonal 27,
    neighbour (dx, dy, dz) -(1 + beta (dx + dy + dz) / 3) (1 + 0.1 xi), xi ~
    U[-1, 1] per entry (nonsymmetric).  The stand-in for Table 2's
    poisson3Db (3D, nonsymmetric, kappa O(10^3)) at g = 44."""
    rng = np.random.default_rng(seed)
    n = g ** 3
    idx = np.arange(n).reshape(g, g, g)
    rows, cols, vals = [idx.ravel()], [idx.ravel()], [np.full(n, 27.0)]
    for dx in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dz in (-1, 0, 1):
                if dx == dy == dz == 0:
                    continue
                src = idx[max(0, -dx):g - max(0, dx), max(0, -dy):g - max(0, dy), max(0, -dz):g - max(0, dz)]
                dst = idx[max(0, dx):g - max(0, -dx), max(0, dy):g - max(0, -dy), max(0, dz):g - max(0, -dz)]
                rows.append(src.ravel())
                cols.append(dst.ravel())
                vals.append(np.full(src.size, -(1.0 + beta * (dx + dy + dz) / 3.0)))
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    off = rows != cols
    vals[off] *= 1.0 + 0.1 * rng.uniform(-1.0, 1.0, size=int(off.sum()))
    return _csr_from_coo(n, rows, cols, vals)


def sparse_random(n: int, nnz_row: int, symmetric: bool = False, dominance: float = 2.0,
                  indefinite: bool = False, seed: int = 0):
    """Random sparsity: every row draws nnz_row - 1 off-diagonal columns
    uniformly (duplicates merged), values N(0,1); symmetric=True draws half as
    many and mirrors the pattern and values ((R + R^T) / 2).  The diagonal is dominance times the
    row's off-diagonal absolute sum (so the matrix is nonsingular and its
    condition number is modest), with a random sign per row if indefinite.
    Stand-ins for Table 2's cage-11 (nonsymmetric, kappa O(1)) and SiO
    (symmetric indefinite)."""
    rng = np.random.default_rng(seed)
    k = (nnz_row - 1) // 2 if symmetric else nnz_row - 1  # mirroring doubles the off-diagonals
    rows = np.repeat(np.arange(n), k)
    cols = rng.integers(0, n - 1, size=n * k)
    cols = cols + (cols >= rows)  # skip the diagonal
    vals = rng.standard_normal(n * k)
    if symmetric:
        rows, cols = np.concatenate([rows, cols]), np.concatenate([cols, rows])
        vals = np.concatenate([vals, vals]) * 0.5
    indptr, indices, data = _csr_from_coo(n, rows, cols, vals)
    rsum = np.add.reduceat(np.abs(data), indptr[:-1])
    sign = rng.choice([-1.0, 1.0], size=n) if indefinite else np.ones(n)
    diag = dominance * np.maximum(rsum, 1.0) * sign
    rows2 = np.concatenate([np.repeat(np.arange(n), np.diff(indptr)), np.arange(n)])
    cols2 = np.concatenate([indices, np.arange(n)])
    return _csr_from_coo(n, rows2, cols2, np.concatenate([data, diag]))


# Table 2 stand-ins with the restart values of Table 3 (m_in, m_out) and m of
# the plain GMRES(m) it is compared with.
SPARSE_CONFIGS = {
    "sio_like": dict(kind="random", n=33401, nnz_row=39, symmetric=True, dominance=1.05, indefinite=True,
                     m_in=30, m_out=20, m=150),
    "cage11_like": dict(kind="random", n=39082, nnz_row=14, symmetric=False, dominance=2.0, indefinite=False,
                        m_in=10, m_out=4, m=18),
    "poisson3db_like": dict(kind="stencil27", g=44, m_in=20, m_out=10, m=50),
}


def sparse_system(name: str, seed: int = 0, scale: float = 1.0):
    """(indptr, indices, data, b, x_true, cfg) for a Table 2 stand-in;
    x_true ~ U[-1, 1] and b = A x_true in FP64 (problem construction).
    scale < 1 shrinks the order (n, or g) for tests."""
    import scipy.sparse as sp
    cfg = dict(SPARSE_CONFIGS[name])
    if cfg["kind"] == "stencil27":
        g = max(3, int(round(cfg["g"] * scale)))
        indptr, indices, data = sparse_stencil27(g, seed=seed)
    else:
        n = max(8, int(round(cfg["n"] * scale)))
        indptr, indices, data = sparse_random(n, min(cfg["nnz_row"], n), cfg["symmetric"], cfg["dominance"],
                                              cfg["indefinite"], seed=seed)
    n = len(indptr) - 1
    rng = np.random.default_rng(seed + 7919)
    x = rng.uniform(-1.0, 1.0, size=n)
    b = sp.csr_matrix((data, indices, indptr), shape=(n, n)) @ x
    return indptr, indices, data, b, x, cfg
