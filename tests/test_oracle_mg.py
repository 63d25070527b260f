"""Pins of the multigrid-preconditioned CG oracle (oracle/mg.py).

Each check is a property the construction must have, so that a plausible
mistake (a wrong interpolation weight, a dropped coupling in a line system,
restriction not the transpose of prolongation, a bad coarse correction)
fails one of them:
* coarsening preserves the total width and keeps an odd last cell;
* prolongation rows sum to one and reproduce a linear function of the cell
  centres between coarse centres exactly;
* the line systems are the diagonal plus the couplings along their axis;
* the V-cycle is symmetric and positive definite on the zero-sum subspace
  (what CG needs of a preconditioner);
* with a single level the V-cycle is the pseudo-inverse and PCG ends in one
  iteration;
* MG-PCG reaches the plain oracle's solution, in a number of iterations that
  does not grow with the grid (8-12 from 32^2 to 256^2, uniform and
  stretched).
"""
import numpy as np
import pytest

import oracle
from oracle import mg
from paper_2604_01800_gb300 import inputs as I


def _ragged(nx, ny, seed):
    g = I.rng(seed)
    return I.random_spacing(nx, g), I.random_spacing(ny, g), g


def test_coarsening_keeps_the_domain():
    w = np.array([1.0, 2.0, 3.0, 4.0, 5.0])
    c = mg.coarsen(w)
    assert np.allclose(c, [3.0, 7.0, 5.0]) and c.sum() == w.sum()
    assert np.allclose(mg.coarsen(np.array([2.5])), [2.5])


@pytest.mark.parametrize("n", [8, 9, 13])
def test_prolongation_is_linear_interpolation(n):
    g = I.rng(n)
    wf = I.random_spacing(n, g)
    wc = mg.coarsen(wf)
    P = mg.prolong_1d(wf, wc).toarray()
    assert np.allclose(P.sum(axis=1), 1.0)
    xf, xc = mg.centres(wf), mg.centres(wc)
    lin = P @ (2.0 + 3.0 * xc)
    # exact wherever the fine centre lies between two coarse centres
    inside = (xf >= xc[0]) & (xf <= xc[-1])
    assert np.allclose(lin[inside], 2.0 + 3.0 * xf[inside], rtol=1e-12, atol=1e-12)
    assert np.all(P >= 0.0)


def test_line_systems_are_the_axis_couplings():
    dx, dy, g = _ragged(7, 6, 3)
    L = mg.Level(dx, dy)
    A = L.A.toarray()
    nx = L.nx
    Tx = np.zeros_like(A)
    Ty = np.zeros_like(A)
    for r in range(A.shape[0]):
        for c in range(A.shape[1]):
            if r == c:
                Tx[r, c] = Ty[r, c] = A[r, c]
            elif r // nx == c // nx and abs(r - c) == 1:
                Tx[r, c] = A[r, c]
            elif r % nx == c % nx and abs(r - c) == nx:
                Ty[r, c] = A[r, c]
    v = g.standard_normal(A.shape[0])
    assert np.allclose(Tx @ L.xline_solve(v), v, atol=1e-12)
    assert np.allclose(Ty @ L.yline_solve(v), v, atol=1e-12)
    assert np.allclose(Tx + Ty - np.diag(np.diag(A)), A)     # together they are A


@pytest.mark.parametrize("shape", [(13, 10), (32, 24), (17, 33)])
def test_vcycle_is_symmetric_positive_definite(shape):
    dx, dy, g = _ragged(*shape, 5)
    M = mg.MGPreconditioner(dx, dy, coarse_cells=16)
    assert len(M.levels) >= 3
    n = shape[0] * shape[1]
    u, v = g.standard_normal(n), g.standard_normal(n)
    u -= u.mean()
    v -= v.mean()
    a, b = u @ M(v), v @ M(u)
    assert abs(a - b) <= 1e-10 * max(abs(a), 1.0)
    for _ in range(5):
        w = g.standard_normal(n)
        w -= w.mean()
        assert w @ M(w) > 0.0


def test_single_level_is_the_pseudo_inverse():
    dx, dy, g = _ragged(9, 7, 8)
    M = mg.MGPreconditioner(dx, dy, coarse_cells=10 ** 6)
    assert len(M.levels) == 1
    A = M.levels[0].A.toarray()
    r = g.standard_normal(A.shape[0])
    r -= r.mean()
    assert np.allclose(A @ M(r), r, atol=1e-10 * np.abs(r).max())
    S = I.gaussian_rhs(dx, dy, g, 3)
    _, info = mg.mgpcg_solve(dx, dy, S, tol_rel=1e-10, coarse_cells=10 ** 6)
    assert info["iters"] <= 1


@pytest.mark.parametrize("case", ["c1", "ragged"])
def test_mgpcg_matches_the_plain_oracle(case):
    if case == "c1":
        w = I.config1(0)
        dx, dy, S = w.dx, w.dy, w.f
    else:
        dx, dy, g = _ragged(45, 38, 11)
        S = I.gaussian_rhs(dx, dy, g, 5)
    x, info = mg.mgpcg_solve(dx, dy, S, tol_rel=1e-10)
    xo, _, _ = oracle.solve(dx, dy, S, tol_rel=1e-11)
    assert info["rel_res_true"] <= 1e-10
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) <= 1e-8
    V = np.outer(dy, dx)
    assert abs((V * x).sum()) <= 1e-12 * (V * np.abs(x)).sum()


@pytest.mark.parametrize("n", [32, 64, 128, 256])
def test_iterations_do_not_grow_with_the_grid(n):
    for dx in (I.uniform_spacing(n), I.tanh_spacing(n, 2.0)):
        S = I.gaussian_rhs(dx, dx, I.rng(n), 6)
        _, info = mg.mgpcg_solve(dx, dx, S, tol_rel=1e-8)
        assert info["iters"] <= 12, (n, info)
