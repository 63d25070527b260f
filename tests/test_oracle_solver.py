"""Pins of the oracle's solve against brute force, a library solver, and the
second-order convergence of the scheme on a manufactured solution."""
import time

import numpy as np
import pytest

import oracle
from paper_2604_01800_gb300 import inputs as I


def _bordered_solve(A, b):
    """Dense LU of [A 1; 1^T 0] [x; l] = [b; 0]: the minimum-sum solution."""
    n = A.shape[0]
    K = np.zeros((n + 1, n + 1))
    K[:n, :n] = A
    K[:n, n] = 1.0
    K[n, :n] = 1.0
    rhs = np.concatenate([b, [0.0]])
    return np.linalg.solve(K, rhs)[:n]


@pytest.mark.parametrize("seed,nx,ny", [(11, 5, 7), (12, 8, 8), (13, 3, 6), (14, 1, 9)])
def test_pcg_matches_dense_bordered_solve(seed, nx, ny):
    g = I.rng(seed)
    dx, dy = g.uniform(0.1, 2.0, nx), g.uniform(0.1, 2.0, ny)
    S = g.standard_normal((ny, nx))
    V = np.outer(dy, dx)
    S -= (V * S).sum() / V.sum()
    x, info, st = oracle.solve(dx, dy, S, tol_rel=1e-13)
    assert st == oracle.OR_OK
    A = oracle.CSR(dx, dy).dense()
    b = oracle.scaled_rhs(dx, dy, S).reshape(-1)
    xd = _bordered_solve(A, b - b.mean()).reshape(ny, nx)
    xd = oracle.volume_mean_free(dx, dy, xd)
    assert np.max(np.abs(x - xd)) <= 1e-10 * np.max(np.abs(xd))


def test_matches_scipy_spsolve():
    import scipy.sparse.linalg as spla
    w = I.config1(3)
    x, info, st = oracle.solve(w.dx, w.dy, w.f, tol_rel=1e-12)
    assert st == oracle.OR_OK and info["rel_res_true"] <= 1e-12
    A = oracle.CSR(w.dx, w.dy).scipy().tolil()
    b = oracle.scaled_rhs(w.dx, w.dy, w.f).reshape(-1)
    b -= b.mean()
    # pin one node to remove the null space, then normalise
    A[0, :] = 0.0
    A[0, 0] = 1.0
    b[0] = 0.0
    xs = spla.spsolve(A.tocsr(), b).reshape(w.ny, w.nx)
    xs = oracle.volume_mean_free(w.dx, w.dy, xs)
    assert np.linalg.norm(x - xs) <= 1e-9 * np.linalg.norm(xs)


def _manufactured_error(dx, dy):
    xc, yc = I.centres(dx), I.centres(dy)
    p = np.outer(np.cos(np.pi * yc), np.cos(np.pi * xc))
    S = -2.0 * np.pi ** 2 * p              # Laplacian of p; Neumann-compatible
    V = np.outer(dy, dx)
    S -= (V * S).sum() / V.sum()
    x, info, st = oracle.solve(dx, dy, S, tol_rel=1e-10)
    assert st == oracle.OR_OK
    pe = oracle.volume_mean_free(dx, dy, p)
    err = x - pe
    return np.sqrt((V * err ** 2).sum()), np.abs(err).max()


@pytest.mark.parametrize("family", ["tanh", "box"])
def test_manufactured_solution_second_order(family):
    errs = []
    ns = [32, 64, 128, 256]
    for n in ns:
        if family == "tanh":
            d = I.tanh_spacing(n, 2.0)
        else:
            # a box grid at n=32 refined by bisecting every cell
            d0 = I.box_spacing(32, 0.4, 0.6, 1.1)
            k = n // 32
            d = np.repeat(d0 / k, k)
        errs.append(_manufactured_error(d, d))
    l2 = np.array([e[0] for e in errs])
    order = np.log2(l2[:-1] / l2[1:])
    assert np.all(order > 1.8) and np.all(order < 2.3), order
    mx = np.array([e[1] for e in errs])
    assert np.all(np.log2(mx[:-1] / mx[1:]) > 1.5)


def test_incompatible_rhs_is_rejected():
    w = I.config1(0)
    S = w.f + 1.0                            # nonzero volume mean
    _, info, st = oracle.solve(w.dx, w.dy, S)
    assert st == oracle.OR_ERR_INCOMPATIBLE and info["incompat"] > 1e-6


def test_zero_rhs_gives_zero():
    w = I.config1(0)
    x, info, st = oracle.solve(w.dx, w.dy, np.zeros_like(w.f), x0=np.ones_like(w.f))
    assert st == oracle.OR_OK and np.all(x == 0.0)


def test_config1_fast_and_accurate():
    w = I.config1(0)
    t0 = time.perf_counter()
    x, info, st = oracle.solve(w.dx, w.dy, w.f, tol_rel=1e-8)
    assert time.perf_counter() - t0 < 1.0
    assert st == oracle.OR_OK and info["rel_res_true"] <= 1e-8
    assert oracle.true_relres(w.dx, w.dy, w.f, x) <= 1e-8
    V = np.outer(w.dy, w.dx)
    assert abs((V * x).sum()) <= 1e-12 * np.abs(V * x).sum()


def test_warm_start_converges_to_same_solution():
    w = I.config1(1)
    x1, _, _ = oracle.solve(w.dx, w.dy, w.f, tol_rel=1e-11)
    x0 = I.rng(7).standard_normal(w.f.shape)
    x2, _, _ = oracle.solve(w.dx, w.dy, w.f, tol_rel=1e-11, x0=x0)
    assert np.linalg.norm(x1 - x2) <= 1e-8 * np.linalg.norm(x1)
