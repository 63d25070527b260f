"""Pins of the oracle's HyDEA solve (Eqs. 11-12 and the CG/DLSM alternation).

The DLSM step is pinned by what the line search must satisfy whatever the
direction.  With the exact error as the direction, alpha = 1 and the
residual vanishes.  For any direction, the new residual is orthogonal to it,
(r - alpha A e) . e = 0 (the step is optimal along e); the A-norm of the
error does not grow; and a constant added to e changes nothing.  The
alternation is pinned by special cases that reduce to known solvers: a map
that returns nothing useful leaves restarted CG(Num_CG) and then plain PCG,
whose result is the plain oracle's; an exact map finishes after the first
DLSM step.
"""
import numpy as np
import pytest

import oracle
from oracle import hybrid as H
from paper_2604_01800_gb300 import inputs as I


def _system(seed=3, nx=12, ny=9):
    g = I.rng(seed)
    dx, dy = g.uniform(0.2, 1.5, nx), g.uniform(0.2, 1.5, ny)
    S = g.standard_normal((ny, nx))
    V = np.outer(dy, dx)
    S -= (V * S).sum() / V.sum()
    return dx, dy, S


def _pinv(A):
    """Pseudo-inverse of the symmetric operator: invert it on the range
    (eigenvalues above the rounding level), zero on the constants."""
    w, Q = np.linalg.eigh(A)
    keep = w > 1e-10 * w.max()
    return (Q[:, keep] / w[keep]) @ Q[:, keep].T


def _pinv_map(dx, dy):
    """Exact inverse on the range: e = A^+ rhat."""
    P = _pinv(oracle.CSR(dx, dy).dense())
    return lambda rh: (P @ rh.reshape(-1)).reshape(rh.shape)


def test_exact_direction_gives_unit_step_and_zero_residual():
    dx, dy, S = _system()
    A = oracle.CSR(dx, dy)
    b = oracle.scaled_rhs(dx, dy, S).reshape(-1)
    b -= b.mean()
    x0 = np.zeros_like(b)
    P = _pinv(A.dense())
    alpha, x1, r1 = H.dlsm_step(A, x0, b, P @ b)
    assert abs(alpha - 1.0) < 1e-10
    assert np.linalg.norm(r1) <= 1e-10 * np.linalg.norm(b)


def test_step_is_optimal_along_e_and_does_not_increase_energy_error():
    dx, dy, S = _system(seed=4)
    A = oracle.CSR(dx, dy)
    Ad = A.dense()
    b = oracle.scaled_rhs(dx, dy, S).reshape(-1)
    b -= b.mean()
    xs = _pinv(Ad) @ b
    g = I.rng(9)
    x = g.standard_normal(b.size)
    x -= x.mean()
    r = b - A.matvec(x)
    for _ in range(5):
        e = g.standard_normal(b.size)
        alpha, x1, r1 = H.dlsm_step(A, x, r, e)
        ec = e - e.mean()
        assert abs(r1 @ ec) <= 1e-10 * np.linalg.norm(r) * np.linalg.norm(ec)
        err0, err1 = x - xs, x1 - xs
        assert err1 @ (Ad @ err1) <= err0 @ (Ad @ err0) * (1 + 1e-12)
        # r1 is the residual of x1
        assert np.linalg.norm(r1 - (b - Ad @ x1)) <= 1e-10 * np.linalg.norm(b)
        x, r = x1, r1


def test_constant_in_direction_changes_nothing():
    dx, dy, S = _system(seed=5)
    A = oracle.CSR(dx, dy)
    b = oracle.scaled_rhs(dx, dy, S).reshape(-1)
    b -= b.mean()
    e = I.rng(2).standard_normal(b.size)
    a1, x1, r1 = H.dlsm_step(A, np.zeros_like(b), b, e)
    a2, x2, r2 = H.dlsm_step(A, np.zeros_like(b), b, e + 1e3)
    assert abs(a1 - a2) <= 1e-12 * abs(a1)
    assert np.allclose(x1, x2, rtol=0, atol=1e-9 * np.abs(x1).max())
    assert np.allclose(r1, r2, rtol=0, atol=1e-9 * np.abs(r1).max())


def test_null_direction_is_skipped():
    dx, dy, S = _system(seed=6)
    A = oracle.CSR(dx, dy)
    b = oracle.scaled_rhs(dx, dy, S).reshape(-1)
    b -= b.mean()
    assert H.dlsm_step(A, np.zeros_like(b), b, np.ones_like(b)) is None    # a constant: e.Ae = 0
    assert H.dlsm_step(A, np.zeros_like(b), b, np.zeros_like(b)) is None


def test_useless_map_reduces_to_restarted_cg_then_pcg():
    w = I.config1(1)
    x_ref, info_ref, st = oracle.solve(w.dx, w.dy, w.f, tol_rel=1e-10)
    x, info = H.hybrid_solve(w.dx, w.dy, w.f, lambda rh: np.zeros_like(rh), tol_rel=1e-10, budget=60)
    assert info["iters_dlsm"] == 0 and info["dlsm_skipped"] >= 1 and info["fell_back"] == 1
    assert info["rel_res_true"] <= 1e-10 * 1.05
    assert np.linalg.norm(x - x_ref) <= 1e-7 * np.linalg.norm(x_ref)
    # before the budget the CG phases restart every Num_CG iterations
    kinds = [k for k, _ in info["history"][:60]]
    assert kinds == ["cg"] * 60


def test_exact_map_converges_after_first_dlsm_step():
    dx, dy, S = _system(seed=7, nx=10, ny=10)
    x, info = H.hybrid_solve(dx, dy, S, _pinv_map(dx, dy), tol_rel=1e-10)
    assert info["iters_pcg"] == 3 and info["iters_dlsm"] == 1
    assert info["rel_res_true"] <= 1e-10
    xr, _, _ = oracle.solve(dx, dy, S, tol_rel=1e-12)
    assert np.linalg.norm(x - xr) <= 1e-8 * np.linalg.norm(xr)


@pytest.mark.parametrize("theta", [0.3, 0.7])
def test_blended_map_reaches_the_plain_solution(theta):
    dx, dy, S = _system(seed=8, nx=14, ny=11)
    A = oracle.CSR(dx, dy).dense()
    M = (1 - theta) * _pinv(A) + theta * np.diag(1.0 / np.diag(A))
    x, info = H.hybrid_solve(dx, dy, S, lambda rh: (M @ rh.reshape(-1)).reshape(rh.shape), tol_rel=1e-10)
    assert info["iters_dlsm"] >= 1 and info["fell_back"] == 0
    assert info["rel_res_true"] <= 1e-10 * 1.05
    xr, _, _ = oracle.solve(dx, dy, S, tol_rel=1e-12)
    assert np.linalg.norm(x - xr) <= 1e-7 * np.linalg.norm(xr)
    # the iteration pattern is CG^3 DLSM^2 repeated (each phase full length)
    kinds = [k for k, _ in info["history"]]
    assert kinds[:5] == ["cg", "cg", "cg", "dlsm", "dlsm"]
