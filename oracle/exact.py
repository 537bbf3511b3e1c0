"""Exact rational arithmetic (``fractions.Fraction``) used to pin the C oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Everything here is the textbook definition computed without rounding, for
tiny matrices (n <= 8): Gaussian elimination with partial pivoting
(Section 2.1: PA = LU, then Ly = Pb, Ux = y), the exact residual b - Ax
(Algorithm 1 step 4), the infinity norm, and closed forms used as
independent pins (tridiagonal Toeplitz LU and inverse, Hilbert inverse).
"""
from __future__ import annotations

from fractions import Fraction
from math import comb


def to_frac_matrix(A):
    return [[Fraction(float(A[i][j])) for j in range(len(A[0]))] for i in range(len(A))]


def gepp(A):
    """Exact PA = LU with partial pivoting: pivot = largest |a_ik| for i >= k,
    ties to the smallest row index.  Returns (L, U, ipiv, info); ipiv 1-based
    LAPACK style; info = first zero-pivot column + 1 (elimination continues)."""
    n = len(A)
    M = [row[:] for row in A]
    ipiv = []
    info = 0
    for k in range(n):
        p = k
        for i in range(k + 1, n):
            if abs(M[i][k]) > abs(M[p][k]):
                p = i
        ipiv.append(p + 1)
        if M[p][k] == 0:
            if info == 0:
                info = k + 1
            continue
        M[k], M[p] = M[p], M[k]
        for i in range(k + 1, n):
            M[i][k] = M[i][k] / M[k][k]
            for j in range(k + 1, n):
                M[i][j] -= M[i][k] * M[k][j]
    L = [[(M[i][j] if j < i else (Fraction(1) if i == j else Fraction(0))) for j in range(n)]
         for i in range(n)]
    U = [[(M[i][j] if j >= i else Fraction(0)) for j in range(n)] for i in range(n)]
    return L, U, ipiv, info


def apply_pivots(b, ipiv):
    b = list(b)
    for k, p in enumerate(ipiv):
        p -= 1
        b[k], b[p] = b[p], b[k]
    return b


def solve(A, b):
    """Exact x = A^{-1} b by Gaussian elimination (Section 2.1)."""
    n = len(A)
    L, U, ipiv, info = gepp(A)
    if info:
        raise ZeroDivisionError("singular")
    y = apply_pivots(b, ipiv)
    for i in range(n):
        y[i] = y[i] - sum(L[i][j] * y[j] for j in range(i))
    x = [Fraction(0)] * n
    for i in reversed(range(n)):
        x[i] = (y[i] - sum(U[i][j] * x[j] for j in range(i + 1, n))) / U[i][i]
    return x


def residual(A, x, b):
    """Exact r = b - A x."""
    n = len(A)
    return [b[i] - sum(A[i][j] * x[j] for j in range(n)) for i in range(n)]


def norm_inf(A):
    return max(sum(abs(v) for v in row) for row in A)


def inverse(A):
    n = len(A)
    cols = [solve(A, [Fraction(int(i == j)) for i in range(n)]) for j in range(n)]
    return [[cols[j][i] for j in range(n)] for i in range(n)]


def cholesky(A):
    """Exact L with A = L L^T is irrational in general; this returns the
    exact LDL^T factors (unit L, diagonal D) instead, from which the Cholesky
    factor is L * sqrt(D)."""
    n = len(A)
    L = [[Fraction(0)] * n for _ in range(n)]
    D = [Fraction(0)] * n
    for j in range(n):
        D[j] = A[j][j] - sum(L[j][k] ** 2 * D[k] for k in range(j))
        L[j][j] = Fraction(1)
        for i in range(j + 1, n):
            L[i][j] = (A[i][j] - sum(L[i][k] * L[j][k] * D[k] for k in range(j))) / D[j]
    return L, D


# ---- closed forms -----------------------------------------------------------

def tridiag_toeplitz(n):
    """T = tridiag(-1, 2, -1) as exact fractions."""
    return [[Fraction(2) if i == j else (Fraction(-1) if abs(i - j) == 1 else Fraction(0))
             for j in range(n)] for i in range(n)]


def tridiag_lu_closed_form(n):
    """For T = tridiag(-1,2,-1): GEPP does no exchanges; with 0-based k,
    u_kk = (k+2)/(k+1), l_{k+1,k} = -(k+1)/(k+2), u_{k,k+1} = -1."""
    ukk = [Fraction(k + 2, k + 1) for k in range(n)]
    lsub = [Fraction(-(k + 1), k + 2) for k in range(n - 1)]
    return ukk, lsub


def tridiag_inverse_closed_form(n):
    """(T^{-1})_{ij} = i (n+1-j) / (n+1) for 1-based i <= j, symmetric."""
    inv = [[Fraction(0)] * n for _ in range(n)]
    for i in range(1, n + 1):
        for j in range(1, n + 1):
            a, b = min(i, j), max(i, j)
            inv[i - 1][j - 1] = Fraction(a * (n + 1 - b), n + 1)
    return inv


def hilbert(n):
    return [[Fraction(1, i + j + 1) for j in range(n)] for i in range(n)]


def hilbert_inverse_closed_form(n):
    """(H_n^{-1})_{ij} = (-1)^{i+j} (i+j+1) C(n+i, n-j-1) C(n+j, n-i-1) C(i+j, i)^2
    with 0-based i, j (all entries integers)."""
    inv = [[0] * n for _ in range(n)]
    for i in range(n):
        for j in range(n):
            v = (i + j + 1) * comb(n + i, n - j - 1) * comb(n + j, n - i - 1) * comb(i + j, i) ** 2
            inv[i][j] = Fraction((-1) ** (i + j) * v)
    return inv
