"""FP64 numpy oracle of the multigrid-preconditioned CG partner.  TEST
INFRASTRUCTURE ONLY (the tests and the benchmark's CPU leg use it).

The paper pairs its DLSM steps with several CG-type methods, MGPCG-4 among
them: CG preconditioned by one multigrid V-cycle per iteration (Sec. 2.6,
Tables 2-3; there an algebraic, smoothed-aggregation hierarchy from PETSc).
On a tensor-product grid the geometric analogue is the one restated here,
step by step, with no fusion:

* Hierarchy.  Level 0 is the grid.  Level l+1 merges neighbouring pairs of
  cells along each axis: coarse width W_I = w_{2I} + w_{2I+1}; an odd last
  cell stays alone; an axis of one cell is not coarsened.  Coarsening stops
  at the first level with at most ``coarse_cells`` cells.
* Operator on every level: the volume-scaled variable-spacing 5-point
  operator A = -V M built from that level's widths (re-discretisation).
* Prolongation P = P_y (x) P_x: along each axis a fine cell takes the linear
  interpolation, in cell-centre coordinates, between its parent and the
  coarse neighbour on its side of the parent's centre, or its parent's value
  when there is no such neighbour (the walls, an unmerged cell).
  Restriction R = P^T, so the V-cycle is symmetric.
* Smoother: alternating damped line Jacobi.  An x sweep solves, for every
  grid row, the tridiagonal system of that row's diagonal and x couplings
  (T_x) and updates z <- z + omega T_x^{-1} (r - A z); a y sweep does the same
  along columns.  Before the coarse correction: x sweep then y sweep; after
  it: y sweep then x sweep.  Line relaxation is what makes the smoother work
  on the stretched cells of these grids, whose couplings differ by the cell
  aspect ratio along the two axes.
* Coarsest level: the minimum-norm solution (pseudo-inverse of the singular
  Neumann operator) of the zero-sum residual.
* PCG: preconditioned CG with z = Vcycle(r), the residual projected to zero
  sum after every update, stopped on the true relative residual, and a zero
  volume-weighted mean for the returned solution (as the plain oracle).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.linalg import solve_banded

from . import CSR, scaled_rhs


def coarsen(w):
    """Widths of the next level: sums of neighbouring pairs (odd tail kept)."""
    w = np.asarray(w, dtype=np.float64)
    n = w.size
    if n == 1:
        return w.copy()
    out = np.zeros((n + 1) // 2)
    out[: n // 2] = w[0:2 * (n // 2):2] + w[1:2 * (n // 2):2]
    if n % 2:
        out[-1] = w[-1]
    return out


def centres(w):
    return np.cumsum(w) - 0.5 * np.asarray(w)


def prolong_1d(wf, wc):
    """1-D prolongation matrix [nf x nc] (see the module text)."""
    nf, nc = wf.size, wc.size
    if nf == nc:
        return sp.identity(nf, format="csr")
    xf, xc = centres(wf), centres(wc)
    rows, cols, vals = [], [], []
    for i in range(nf):
        par = i // 2
        nb = par - 1 if xf[i] < xc[par] else par + 1
        if xf[i] == xc[par] or nb < 0 or nb >= nc:
            rows.append(i)
            cols.append(par)
            vals.append(1.0)
            continue
        t = (xf[i] - xc[par]) / (xc[nb] - xc[par])
        rows += [i, i]
        cols += [par, nb]
        vals += [1.0 - t, t]
    return sp.csr_matrix((vals, (rows, cols)), shape=(nf, nc))


class Level:
    def __init__(self, dx, dy):
        self.dx, self.dy = np.asarray(dx, np.float64), np.asarray(dy, np.float64)
        self.nx, self.ny = self.dx.size, self.dy.size
        self.A = CSR(self.dx, self.dy).scipy().tocsr()
        self.diag = self.A.diagonal().copy()
        # line systems: T_x couples cells of a row along x, T_y of a column along y
        fx = np.zeros(self.nx + 1)
        fx[1:-1] = 2.0 / (self.dx[:-1] + self.dx[1:])
        fy = np.zeros(self.ny + 1)
        fy[1:-1] = 2.0 / (self.dy[:-1] + self.dy[1:])
        self.fx, self.fy = fx, fy

    def xline_solve(self, rhs):
        """T_x^{-1} rhs, row by row (rhs [ny*nx])."""
        R = rhs.reshape(self.ny, self.nx)
        out = np.empty_like(R)
        D = self.diag.reshape(self.ny, self.nx)
        for j in range(self.ny):
            ab = np.zeros((3, self.nx))
            ab[0, 1:] = -self.dy[j] * self.fx[1:-1]           # super-diagonal
            ab[1, :] = D[j]
            ab[2, :-1] = -self.dy[j] * self.fx[1:-1]          # sub-diagonal
            out[j] = solve_banded((1, 1), ab, R[j])
        return out.reshape(-1)

    def yline_solve(self, rhs):
        """T_y^{-1} rhs, column by column."""
        R = rhs.reshape(self.ny, self.nx)
        out = np.empty_like(R)
        D = self.diag.reshape(self.ny, self.nx)
        for i in range(self.nx):
            ab = np.zeros((3, self.ny))
            ab[0, 1:] = -self.dx[i] * self.fy[1:-1]
            ab[1, :] = D[:, i]
            ab[2, :-1] = -self.dx[i] * self.fy[1:-1]
            out[:, i] = solve_banded((1, 1), ab, R[:, i])
        return out.reshape(-1)


def hierarchy(dx, dy, coarse_cells=256):
    """The list of levels, finest first, and the prolongations between them."""
    levels, prolongs = [Level(dx, dy)], []
    while levels[-1].nx * levels[-1].ny > coarse_cells and (levels[-1].nx > 1 or levels[-1].ny > 1):
        f = levels[-1]
        c = Level(coarsen(f.dx), coarsen(f.dy))
        prolongs.append(sp.kron(prolong_1d(f.dy, c.dy), prolong_1d(f.dx, c.dx), format="csr"))
        levels.append(c)
    return levels, prolongs


def pseudo_inverse(A):
    """Moore-Penrose inverse of a symmetric matrix from its eigen-decomposition
    (eigenvalues below 1e-12 of the largest count as zero)."""
    lam, V = np.linalg.eigh(A)
    keep = lam > 1e-12 * np.abs(lam).max()
    return (V[:, keep] / lam[keep]) @ V[:, keep].T


class MGPreconditioner:
    def __init__(self, dx, dy, omega=0.8, coarse_cells=256):
        self.levels, self.P = hierarchy(dx, dy, coarse_cells)
        self.omega = omega
        self.coarse_pinv = pseudo_inverse(self.levels[-1].A.toarray())

    def xsweep(self, L, r, z):
        return z + self.omega * L.xline_solve(r - L.A @ z)

    def ysweep(self, L, r, z):
        return z + self.omega * L.yline_solve(r - L.A @ z)

    def vcycle(self, r, level=0):
        L = self.levels[level]
        if level == len(self.levels) - 1:
            return self.coarse_pinv @ (r - r.mean())
        z = self.xsweep(L, r, np.zeros_like(r))
        z = self.ysweep(L, r, z)
        rc = self.P[level].T @ (r - L.A @ z)
        z = z + self.P[level] @ self.vcycle(rc, level + 1)
        z = self.ysweep(L, r, z)
        return self.xsweep(L, r, z)

    def __call__(self, r):
        return self.vcycle(np.asarray(r, np.float64).reshape(-1))


def mgpcg_solve(dx, dy, S, tol_rel=1e-8, x0=None, maxit=10000, omega=0.8, coarse_cells=256):
    """Solve M x = S with multigrid-preconditioned CG; returns (x, info)."""
    dx, dy = np.asarray(dx, np.float64), np.asarray(dy, np.float64)
    nx, ny = dx.size, dy.size
    M = MGPreconditioner(dx, dy, omega, coarse_cells)
    A = M.levels[0].A
    b = scaled_rhs(dx, dy, S).reshape(-1)
    b = b - b.mean()
    bn = np.linalg.norm(b)
    x = np.zeros(nx * ny) if x0 is None else np.asarray(x0, np.float64).reshape(-1).copy()
    r = b - A @ x
    r -= r.mean()
    it = 0
    if bn > 0 and np.linalg.norm(r) > tol_rel * bn:
        z = M(r)
        p = z.copy()
        rz = r @ z
        while it < maxit:
            q = A @ p
            alpha = rz / (p @ q)
            x += alpha * p
            r -= alpha * q
            r -= r.mean()
            it += 1
            if np.linalg.norm(r) <= tol_rel * bn:
                rt = b - A @ x                 # confirm with the true residual
                rt -= rt.mean()
                if np.linalg.norm(rt) <= tol_rel * bn:
                    break
                r = rt
            z = M(r)
            rz_new = r @ z
            p = z + (rz_new / rz) * p
            rz = rz_new
    rt = b - A @ x
    rt -= rt.mean()
    V = np.outer(dy, dx).reshape(-1)
    x -= (V * x).sum() / V.sum()
    return x.reshape(ny, nx), {"iters": it, "rel_res_true": float(np.linalg.norm(rt) / bn) if bn > 0 else 0.0,
                               "levels": len(M.levels)}
