"""Pins of the projection-step oracle (oracle/projection.py, Sec. 2.1 Eqs. 6-8).

* D G is the PPE operator: -V (D G p) equals the assembled A p of the PPE
  oracle, for random p on stretched grids (so D, G and the PPE agree on the
  face geometry, signs and walls).
* A projected field is discretely divergence-free: with dp from the PPE
  oracle for S = D u* / dt, the interior divergence of u - dt G dp is zero to
  the solve's tolerance.
* Closed forms: G of a linear function is its constant slope on interior
  faces; D of a linear face field is exact; on uniform grids D converges at
  second order for a smooth field.
"""
import numpy as np
import pytest

import oracle
from oracle import projection as PJ
from paper_2604_01800_gb300 import inputs as I


def _grid(nx, ny, seed):
    g = I.rng(seed)
    return I.random_spacing(nx, g), I.random_spacing(ny, g), g


@pytest.mark.parametrize("shape", [(7, 5), (33, 20)])
def test_dg_is_the_ppe_operator(shape):
    dx, dy, g = _grid(*shape, 3)
    p = g.standard_normal((shape[1], shape[0]))
    gu, gv = PJ.gradient(dx, dy, p)
    Mp = PJ.divergence(dx, dy, gu, gv)
    Ap = oracle.apply(dx, dy, p)
    assert np.allclose(-np.outer(dy, dx) * Mp, Ap, rtol=1e-12, atol=1e-12 * np.abs(Ap).max())


def test_projected_field_is_divergence_free():
    dx, dy, g = _grid(40, 30, 5)
    u = g.standard_normal((30, 41))
    v = g.standard_normal((31, 40))
    u[:, 0] = u[:, -1] = 0.0             # walls at rest: no normal flow
    v[0, :] = v[-1, :] = 0.0
    dt = 0.01
    S = PJ.ppe_source(dx, dy, u, v, dt)
    dp, info, st = oracle.solve(dx, dy, S, tol_rel=1e-12)
    assert st == 0
    un, vn, _ = PJ.project(dx, dy, u, v, np.zeros_like(dp), dp, dt)
    div = PJ.divergence(dx, dy, un, vn)
    assert np.abs(div).max() <= 1e-9 * np.abs(PJ.divergence(dx, dy, u, v)).max()
    assert np.allclose(un[:, [0, -1]], 0.0) and np.allclose(vn[[0, -1], :], 0.0)


def test_inflow_outflow_walls():
    """A stream through the left and right walls (equal fluxes): the source
    carries the wall fluxes, is compatible, and the projected field is
    divergence free with the wall velocities unchanged."""
    dx, dy, g = _grid(36, 24, 9)
    u = 1.0 + 0.1 * g.standard_normal((24, 37))
    v = 0.1 * g.standard_normal((25, 36))
    u[:, -1] = u[:, 0] * 1.0                    # outflow profile = inflow profile
    v[0, :] = v[-1, :] = 0.0
    dt = 0.02
    S = PJ.ppe_source(dx, dy, u, v, dt)
    V = np.outer(dy, dx)
    assert abs((V * S).sum()) <= 1e-12 * (V * np.abs(S)).sum()
    dp, info, st = oracle.solve(dx, dy, S, tol_rel=1e-12)
    un, vn, _ = PJ.project(dx, dy, u, v, np.zeros_like(dp), dp, dt)
    assert np.abs(PJ.divergence(dx, dy, un, vn)).max() <= 1e-9 * np.abs(PJ.divergence(dx, dy, u, v)).max()
    assert np.array_equal(un[:, [0, -1]], u[:, [0, -1]])


def test_closed_forms():
    dx, dy, g = _grid(12, 9, 7)
    xc = np.cumsum(dx) - 0.5 * dx
    yc = np.cumsum(dy) - 0.5 * dy
    p = 2.0 * xc[None, :] - 3.0 * yc[:, None] + 1.0
    gu, gv = PJ.gradient(dx, dy, p)
    assert np.allclose(gu[:, 1:-1], 2.0) and np.allclose(gv[1:-1, :], -3.0)
    xf = np.concatenate([[0.0], np.cumsum(dx)])
    yf = np.concatenate([[0.0], np.cumsum(dy)])
    u = np.tile(0.5 * xf, (9, 1))
    v = np.tile(4.0 * yf[:, None], (1, 12))
    assert np.allclose(PJ.divergence(dx, dy, u, v), 4.5)


def test_divergence_is_second_order_on_uniform_grids():
    errs = []
    for n in (16, 32, 64):
        d = I.uniform_spacing(n)
        xf = np.linspace(0.0, 1.0, n + 1)
        xc = (np.arange(n) + 0.5) / n
        u = np.sin(np.pi * xf)[None, :] * np.cos(np.pi * xc)[:, None]
        v = np.cos(np.pi * xc)[None, :] * np.sin(np.pi * xf)[:, None]
        exact = 2.0 * np.pi * np.cos(np.pi * xc)[None, :] * np.cos(np.pi * xc)[:, None]
        errs.append(np.abs(PJ.divergence(d, d, u, v) - exact).max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all((orders > 1.8) & (orders < 2.2)), orders
