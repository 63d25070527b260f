"""FP64 HyDEA solve: Jacobi PCG phases alternating with DLSM steps.
TEST INFRASTRUCTURE ONLY (see the package docstring).

Written from the paper's method description (Sec. 2.2):

* DLSM step (Eqs. 11-12): the direction e comes from a learned map applied
  to the current residual.  The step length that minimises the A-norm of the
  error along e is alpha = (r . e) / (e . A e); then x <- x + alpha e and
  r <- r - alpha A e.
* The solve alternates up to Num_CG iterations of Jacobi PCG with up to
  Num_DLSM DLSM steps, and tests convergence after every single iteration of
  either kind.

Readings where the paper is silent (they are the readings the library
documents, restated here independently):

* Each CG-type phase is a fresh Jacobi PCG start from the current x and the
  current residual: z = D^-1 r, p = z.
* The map receives r / ||r|| (its input scale is free; alpha absorbs it).
* The constant part of e is removed before alpha is formed (A 1 = 0, so it
  does not change the iteration in exact arithmetic).
* A step whose curvature e . A e is not positive beyond a relative guard is
  skipped and the next CG phase begins.
* After `budget` iterations in total the solve continues as plain PCG.
* The residual is kept orthogonal to the constants (singular Neumann system).

Plain numpy on the oracle's assembled CSR operator; no blocking, no fusion.
"""
from __future__ import annotations

import numpy as np

from . import CSR, scaled_rhs


def dlsm_step(A: CSR, x, r, e, guard=1e-10, diag_max=None):
    """One DLSM step (Eqs. 11-12) on flat FP64 vectors.  Returns
    (alpha, x_new, r_new), or None when the curvature guard rejects e."""
    e = np.asarray(e, dtype=np.float64).reshape(-1)
    e = e - e.mean()
    q = A.matvec(e)
    eq = float(e @ q)
    ee = float(e @ e)
    if diag_max is None:
        diag_max = float(np.max(_diag(A)))
    if not eq > guard * ee * diag_max:
        return None
    alpha = float(r @ e) / eq
    return alpha, x + alpha * e, r - alpha * q


def _diag(A: CSR):
    d = np.zeros(A.n)
    for row in range(A.n):
        for k in range(A.rowptr[row], A.rowptr[row + 1]):
            if A.col[k] == row:
                d[row] = A.val[k]
    return d


def hybrid_solve(dx, dy, S, direction, tol_rel=1e-8, num_cg=3, num_dlsm=2, budget=20000, maxit=200000,
                 guard=1e-10):
    """Solve M x = S with HyDEA.  `direction(rhat)` maps a unit-norm residual
    field [ny, nx] to a direction field [ny, nx].  Returns (x [ny, nx] with
    zero volume-weighted mean, info dict)."""
    dx = np.asarray(dx, dtype=np.float64)
    dy = np.asarray(dy, dtype=np.float64)
    nx, ny = dx.size, dy.size
    A = CSR(dx, dy)
    dinv = 1.0 / _diag(A)
    diag_max = float(np.max(1.0 / dinv))
    b = scaled_rhs(dx, dy, S).reshape(-1)
    b = b - b.mean()
    bnorm = float(np.linalg.norm(b))
    x = np.zeros(nx * ny)
    r = b.copy()
    it_pcg = it_dlsm = skipped = 0
    fell_back = False
    history = []

    def converged():
        return float(np.linalg.norm(r)) <= tol_rel * bnorm

    def total():
        return it_pcg + it_dlsm

    while bnorm > 0 and not converged() and total() < maxit + budget:
        # CG-type phase: a fresh Jacobi PCG start from the current x
        z = dinv * r
        p = z.copy()
        rz = float(r @ z)
        k = 0
        while k < num_cg or fell_back:
            q = A.matvec(p)
            alpha = rz / float(p @ q)
            x += alpha * p
            r -= alpha * q
            r -= r.mean()
            it_pcg += 1
            k += 1
            history.append(("cg", float(np.linalg.norm(r)) / bnorm))
            if converged() or total() >= maxit + budget:
                break
            if not fell_back and total() >= budget:
                fell_back = True
            z = dinv * r
            rz_new = float(r @ z)
            p = z + (rz_new / rz) * p
            rz = rz_new
        if converged() or fell_back:
            continue
        # DLSM phase
        for _ in range(num_dlsm):
            rhat = (r / np.linalg.norm(r)).reshape(ny, nx)
            step = dlsm_step(A, x, r, direction(rhat), guard=guard, diag_max=diag_max)
            if step is None:
                skipped += 1
                break
            _, x, r = step
            r -= r.mean()
            it_dlsm += 1
            history.append(("dlsm", float(np.linalg.norm(r)) / bnorm))
            if converged():
                break
            if total() >= budget:
                fell_back = True
                break

    xf = x.reshape(ny, nx)
    V = np.outer(dy, dx)
    xf = xf - (V * xf).sum() / V.sum()
    rt = b - A.matvec(xf)
    rt -= rt.mean()
    info = {"iters_pcg": it_pcg, "iters_dlsm": it_dlsm, "dlsm_skipped": skipped, "fell_back": int(fell_back),
            "rel_res_true": float(np.linalg.norm(rt)) / bnorm if bnorm > 0 else 0.0, "history": history}
    return xf, info
