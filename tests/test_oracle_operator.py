"""Pins of the oracle's operator A = -V M against what the mathematics fixes.

* On a uniform n x n grid of [0,1]^2 the scaled operator is the unit-weight
  graph Laplacian with Neumann walls, diagonalised by the DCT-II basis
  cos(pi k (i+1/2)/n) cos(pi l (j+1/2)/n) with eigenvalues
  4 sin^2(pi k / 2n) + 4 sin^2(pi l / 2n).  A wrong face coefficient, a
  transposed index or a wrong wall treatment breaks this identity.
* Symmetry (exact, bitwise), zero row sums (constant null space),
  positive semidefiniteness with a one-dimensional null space.
"""
import numpy as np
import pytest

import oracle
from paper_2604_01800_gb300 import inputs as I


@pytest.mark.parametrize("n", [8, 13, 32])
def test_dct_eigenpairs_uniform(n):
    dx = dy = I.uniform_spacing(n)
    A = oracle.CSR(dx, dy)
    i = np.arange(n) + 0.5
    for k, l in [(0, 1), (1, 0), (1, 1), (3, 2), (n - 1, n - 1), (n // 2, 1)]:
        v = np.outer(np.cos(np.pi * l * i / n), np.cos(np.pi * k * i / n))
        lam = 4 * np.sin(np.pi * k / (2 * n)) ** 2 + 4 * np.sin(np.pi * l / (2 * n)) ** 2
        Av = A.matvec(v).reshape(n, n)
        assert np.max(np.abs(Av - lam * v)) <= 1e-13 * max(1.0, lam)


def test_dct_eigenpairs_rectangle():
    nx, ny, lx, ly = 12, 7, 2.0, 1.0
    dx, dy = I.uniform_spacing(nx, lx), I.uniform_spacing(ny, ly)
    hx, hy = lx / nx, ly / ny
    A = oracle.CSR(dx, dy)
    i, j = np.arange(nx) + 0.5, np.arange(ny) + 0.5
    for k, l in [(1, 0), (2, 3), (11, 6)]:
        v = np.outer(np.cos(np.pi * l * j / ny), np.cos(np.pi * k * i / nx))
        # scaled rows: dy/dx * (2 - 2cos) in x, dx/dy * (2 - 2cos) in y
        lam = (hy / hx) * 4 * np.sin(np.pi * k / (2 * nx)) ** 2 + (hx / hy) * 4 * np.sin(np.pi * l / (2 * ny)) ** 2
        assert np.allclose(A.matvec(v).reshape(ny, nx), lam * v, atol=1e-13, rtol=0)


def _random_grid(seed, nx, ny):
    g = I.rng(seed)
    return g.uniform(0.2, 3.0, nx), g.uniform(0.2, 3.0, ny)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_symmetric_bitwise_and_zero_row_sums(seed):
    dx, dy = _random_grid(seed, 9, 6)
    A = oracle.CSR(dx, dy).dense()
    assert np.array_equal(A, A.T)
    scale = np.abs(A).max()
    assert np.max(np.abs(A.sum(axis=1))) <= 1e-15 * scale * 8


@pytest.mark.parametrize("seed", [4, 5])
def test_psd_with_constant_null_space(seed):
    dx, dy = _random_grid(seed, 7, 8)
    A = oracle.CSR(dx, dy).dense()
    w = np.linalg.eigvalsh(A)
    assert w[0] >= -1e-12 * w[-1]
    assert abs(w[0]) <= 1e-12 * w[-1]
    assert w[1] > 1e-6 * w[-1]            # connected grid: null space is 1-D


def test_stencil_entries_match_definition():
    """Off-diagonals of one interior row equal -dy*2/(dx_i+dx_{i+1}) and
    -dx*2/(dy_j+dy_{j+1}) (Sec. 2.1 staggered-grid D and G)."""
    dx = np.array([0.1, 0.2, 0.4, 0.3])
    dy = np.array([0.5, 0.25, 0.25])
    A = oracle.CSR(dx, dy).dense()
    i, j = 1, 1
    r = j * 4 + i
    assert A[r, r + 1] == -dy[j] * 2 / (dx[i] + dx[i + 1])
    assert A[r, r - 1] == -dy[j] * 2 / (dx[i - 1] + dx[i])
    assert A[r, r + 4] == -dx[i] * 2 / (dy[j] + dy[j + 1])
    assert A[r, r - 4] == -dx[i] * 2 / (dy[j - 1] + dy[j])
    # wall rows have no flux through the wall
    assert np.count_nonzero(A[0]) == 3
