"""Algorithm 2 (Section 2.2): the mixed-precision inner-outer iterative method
FGMRES(m_out)-GMRES_SP(m_in) on a sparse matrix in CSR form.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``): only ``tests/``,
``__graft_entry__.smoke()`` and the benchmark's CPU legs may import this
module.  It shares no code with the CUDA library.

Plain numpy, written from the algorithm as the paper states it:

  outer loop (FP64, flexible GMRES):
      r = b - A x_i;  beta = ||r||_2;  stop if x_i is accurate enough;
      for k = 1 .. m_out:
          v_k = r / h_{k,k-1}                                  (h_{1,0} = beta)
          z_k = one cycle of GMRES_SP(m_in) for A z = v_k, from z = 0
          r = A z_k;  for j = 1 .. k: h_jk = r^T v_j, r = r - h_jk v_j
          h_{k+1,k} = ||r||_2
      y = argmin ||beta e_1 - H_k y||_2;  x_{i+1} = x_i + Z_k y
  inner cycle (working precision T): the same Arnoldi process without a
      preconditioner (textbook GMRES): matrix values and right-hand side
      rounded to T, every operation in T.

The small least-squares problem is solved with Givens rotations and back
substitution (the residual estimate |g_{k+1}| comes with each rotation).
Readings where the paper is silent (they are the library's too):
  * accuracy test at the start of every outer cycle: every column's normwise
    backward error ||r||inf / (||A||inf ||x||inf + ||b||inf) <= tol;
  * "checks for convergence at every inner iteration": the outer cycle ends
    early once the residual estimate |g_{k+1}| <= 0.5 tol (||A||inf xs +
    ||b||inf), xs = max(||x_i||inf, ||b||inf / ||A||inf) (the 2-norm bounds
    the inf-norm, so the next accuracy test is then expected to pass);
  * the inner cycle runs its m_in steps, ending early only at breakdown
    (h_{j+1,j} = 0) or once its estimate is at the working precision's level
    (|g_{j+1}| <= 4 u_T beta_in), where further steps add rounding noise only.
"""
from __future__ import annotations

import numpy as np


def csr_matvec(indptr, indices, data, x):
    """y = A x for A in CSR form: y_i = sum of a_ij x_j over the stored
    entries of row i, in the precision of data and x (every row non-empty)."""
    prod = data * x[indices]
    return np.add.reduceat(prod, indptr[:-1])


def norm_inf_csr(indptr, data):
    """||A||inf: the largest row sum of |a_ij|."""
    return float(np.max(np.add.reduceat(np.abs(data.astype(np.float64)), indptr[:-1])))


def _rotation(a, b):
    """Givens rotation (c, s) with c a + s b = hypot(a, b), -s a + c b = 0."""
    r = np.hypot(a, b)
    if r == 0:
        return a.dtype.type(1), a.dtype.type(0)
    return a / r, b / r


def arnoldi_cycle(matvec, r0, m, dtype, stop_abs=0.0, stop_rel=0.0, precond=None):
    """One cycle of (flexible) GMRES(m) for A z = r0 from z = 0 in precision
    dtype: Arnoldi with modified Gram-Schmidt, Givens rotations on the
    Hessenberg matrix, then z = Z y (Z = the preconditioned basis vectors, or
    V when precond is None).  Ends after m steps, at breakdown, or when the
    residual estimate |g_{j+1}| <= max(stop_abs, stop_rel * beta).
    Returns dict(z, steps, est (estimates after each step), beta, V, Z, H)."""
    r0 = np.asarray(r0).astype(dtype)
    n = r0.shape[0]
    beta = np.sqrt(np.dot(r0, r0)).astype(dtype)
    out = dict(z=np.zeros(n, dtype), steps=0, est=[], beta=float(beta), V=[], Z=[], H=None)
    if beta == 0:
        return out
    V = [r0 / beta]
    Z = []
    H = np.zeros((m + 1, m), dtype)
    R = np.zeros((m + 1, m), dtype)  # H with the rotations applied
    g = np.zeros(m + 1, dtype)
    g[0] = beta
    cs = np.zeros(m, dtype)
    sn = np.zeros(m, dtype)
    steps = 0
    limit = max(float(stop_abs), float(stop_rel) * float(beta))
    for j in range(m):
        zj = V[j] if precond is None else np.asarray(precond(V[j])).astype(dtype)
        Z.append(zj)
        w = np.asarray(matvec(zj)).astype(dtype)
        for i in range(j + 1):  # modified Gram-Schmidt
            H[i, j] = np.dot(w, V[i])
            w = w - H[i, j] * V[i]
        H[j + 1, j] = np.sqrt(np.dot(w, w))
        col = H[: j + 2, j].copy()
        for i in range(j):  # earlier rotations
            a, b = col[i], col[i + 1]
            col[i] = cs[i] * a + sn[i] * b
            col[i + 1] = -sn[i] * a + cs[i] * b
        cs[j], sn[j] = _rotation(col[j], col[j + 1])
        col[j] = cs[j] * col[j] + sn[j] * col[j + 1]
        col[j + 1] = 0
        R[: j + 2, j] = col
        g[j + 1] = -sn[j] * g[j]
        g[j] = cs[j] * g[j]
        steps = j + 1
        out["est"].append(float(abs(g[j + 1])))
        if H[j + 1, j] == 0 or abs(float(g[j + 1])) <= limit:
            break
        V.append(w / H[j + 1, j])
    # back substitution R y = g
    y = np.zeros(steps, dtype)
    for i in range(steps - 1, -1, -1):
        acc = g[i]
        for l in range(i + 1, steps):
            acc = acc - R[i, l] * y[l]
        y[i] = acc / R[i, i]
    z = np.zeros(n, dtype)
    for i in range(steps):
        z = z + y[i] * Z[i]
    out.update(z=z, steps=steps, V=V, Z=Z, H=H[: steps + 1, :steps])
    return out


def gmres_cycle(indptr, indices, data, v, m, dtype=np.float32):
    """One cycle of GMRES_SP(m_in) (dtype float32) or GMRES_DP (float64) for
    A z = v from z = 0, with A's values and v rounded to dtype; the early end
    at the working precision's level as in the module docstring."""
    Ad = np.asarray(data).astype(dtype)
    u = float(np.finfo(dtype).eps) / 2.0
    return arnoldi_cycle(lambda x: csr_matvec(indptr, indices, Ad, x), v, m, dtype, stop_rel=4.0 * u)


def fgmres(indptr, indices, data, b, m_out, m_in, inner=np.float32, tol=1e-14, max_cycles=100,
           inner_solve=None):
    """Algorithm 2: FGMRES(m_out) in FP64 whose preconditioner is one cycle of
    GMRES(m_in) in precision `inner` (float32: GMRES_SP; float64: the
    FGMRES-GMRES_DP comparison).  inner_solve(v) -> z replaces the inner cycle
    (for tests).  Returns dict(x, converged, cycles, outer_steps, inner_steps,
    bwd, hist)."""
    data64 = np.asarray(data, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    n = b.shape[0]
    anorm = norm_inf_csr(indptr, data64)
    bnorm = float(np.max(np.abs(b))) if n else 0.0
    if inner_solve is None:
        def inner_solve(v):
            res = gmres_cycle(indptr, indices, data, v, m_in, inner)
            inner_solve.steps += res["steps"]
            return res["z"]
        inner_solve.steps = 0
    x = np.zeros(n)
    hist = []
    cycles = outer_steps = 0
    converged = False
    while True:
        r = b - csr_matvec(indptr, indices, data64, x)
        xnorm = float(np.max(np.abs(x))) if n else 0.0
        den = anorm * xnorm + bnorm
        bwd = float(np.max(np.abs(r))) / den if den > 0 else 0.0
        hist.append(bwd)
        if bwd <= tol:
            converged = True
            break
        if cycles >= max_cycles:
            break
        xs = max(xnorm, bnorm / anorm) if anorm > 0 else xnorm
        tau = 0.5 * tol * (anorm * xs + bnorm)
        res = arnoldi_cycle(lambda u: csr_matvec(indptr, indices, data64, u), r, m_out, np.float64,
                            stop_abs=tau, precond=lambda v: np.asarray(inner_solve(v), dtype=np.float64))
        x = x + res["z"]
        outer_steps += res["steps"]
        cycles += 1
    return dict(x=x, converged=converged, cycles=cycles, outer_steps=outer_steps,
                inner_steps=getattr(inner_solve, "steps", None), bwd=bwd, hist=hist)


def gmres_restarted(indptr, indices, data, b, m, tol=1e-14, max_cycles=200):
    """Plain restarted GMRES(m) in FP64 (the paper's double-precision
    comparison in Fig. 5, right), with the same accuracy test and the same
    early end of a cycle as the outer loop of fgmres."""
    data64 = np.asarray(data, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    n = b.shape[0]
    anorm = norm_inf_csr(indptr, data64)
    bnorm = float(np.max(np.abs(b))) if n else 0.0
    x = np.zeros(n)
    cycles = steps = 0
    converged = False
    hist = []
    while True:
        r = b - csr_matvec(indptr, indices, data64, x)
        xnorm = float(np.max(np.abs(x))) if n else 0.0
        den = anorm * xnorm + bnorm
        bwd = float(np.max(np.abs(r))) / den if den > 0 else 0.0
        hist.append(bwd)
        if bwd <= tol:
            converged = True
            break
        if cycles >= max_cycles:
            break
        xs = max(xnorm, bnorm / anorm) if anorm > 0 else xnorm
        tau = 0.5 * tol * (anorm * xs + bnorm)
        res = arnoldi_cycle(lambda u: csr_matvec(indptr, indices, data64, u), r, m, np.float64, stop_abs=tau)
        x = x + res["z"]
        steps += res["steps"]
        cycles += 1
    return dict(x=x, converged=converged, cycles=cycles, steps=steps, bwd=bwd, hist=hist)
