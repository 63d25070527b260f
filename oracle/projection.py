"""FP64 numpy oracle of the projection step around the PPE.  TEST
INFRASTRUCTURE ONLY.

The fractional-step method of Sec. 2.1 solves, per time step,
  (6)  dt D G dp = D u* - bc2      (the PPE, M = D G, source S = (D u* - bc2) / dt)
  (7)  u^{n+1} = u* - dt G dp
  (8)  p^{n+1} = p^n + dp
on a staggered (MAC) grid: pressure at cell centres, the x velocity u on the
x faces (i - 1/2, j), the y velocity v on the y faces (i, j - 1/2).

* D (divergence) of a face field at cell (i, j):
  (u[j, i+1] - u[j, i]) / dx_i + (v[j+1, i] - v[j, i]) / dy_j,
  with u of shape [ny, nx+1] and v of shape [ny+1, nx].  The wall faces hold
  the prescribed normal velocity.  Eq. 6 writes the divergence of u* as the
  part D u* over the unknown (interior) faces and the known part from the
  wall faces, bc2; the source the PPE needs so that u^{n+1} is divergence
  free, walls included, is the whole divergence of u*.  It is compatible
  (zero volume-weighted sum) when the net flux through the walls vanishes.
* G (gradient) on the interior faces: (p[j, i] - p[j, i-1]) / ((dx_{i-1} + dx_i) / 2)
  and likewise in y; the wall faces are not updated (their normal velocity
  is prescribed), which is what makes dp's boundary condition homogeneous
  Neumann.
* D G is then exactly the operator M the PPE oracle assembles.
"""
from __future__ import annotations

import numpy as np


def divergence(dx, dy, u, v):
    """D applied to the face field (u [ny, nx+1], v [ny+1, nx]); [ny, nx]."""
    dx, dy = np.asarray(dx, np.float64), np.asarray(dy, np.float64)
    return (u[:, 1:] - u[:, :-1]) / dx[None, :] + (v[1:, :] - v[:-1, :]) / dy[:, None]


def gradient(dx, dy, p):
    """G p on the interior faces (wall faces zero): (gu [ny, nx+1], gv [ny+1, nx])."""
    dx, dy = np.asarray(dx, np.float64), np.asarray(dy, np.float64)
    ny, nx = p.shape
    gu = np.zeros((ny, nx + 1))
    gv = np.zeros((ny + 1, nx))
    gu[:, 1:-1] = (p[:, 1:] - p[:, :-1]) / (0.5 * (dx[:-1] + dx[1:]))[None, :]
    gv[1:-1, :] = (p[1:, :] - p[:-1, :]) / (0.5 * (dy[:-1] + dy[1:]))[:, None]
    return gu, gv


def ppe_source(dx, dy, u, v, dt):
    """The PPE source of Eq. 6 divided by dt: the divergence of u*, the wall
    faces' prescribed normal velocity included."""
    return divergence(dx, dy, np.asarray(u, np.float64), np.asarray(v, np.float64)) / dt


def project(dx, dy, u, v, p, dp, dt):
    """Eqs. 7-8: (u - dt G dp, v - dt G dp, p + dp) on the interior faces."""
    gu, gv = gradient(dx, dy, dp)
    return u - dt * gu, v - dt * gv, p + dp
