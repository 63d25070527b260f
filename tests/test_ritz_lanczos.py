"""The Lanczos / Ritz-vector data recipe of Sec. 2.3 (Eqs. 13-15), on the CPU.

``train.ritz_vectors`` runs m Lanczos steps with full reorthogonalisation on
the grid's operator and returns the Ritz pairs of T_m = V_m^T A V_m.  It is
pinned here against the closed-form spectrum of the operator on a uniform
n x n grid with h = 1/n: A = -V M has the DCT-II eigenvectors
cos(pi k (i + 1/2) / n) cos(pi l (j + 1/2) / n) with eigenvalues
4 [sin^2(pi k / 2n) + sin^2(pi l / 2n)].  With more Lanczos steps than the
start vector has distinct eigenvalues in range(A), the process ends early and
the Ritz values are exactly those eigenvalues: every Ritz value is one of the
closed-form values, and the extreme ones are found.  The operator is applied
by the FP64 oracle (a stand-in for the library's ppe_apply), so this runs
without a GPU.  ``train.ritz_samples`` (Eqs. 14-15) is checked for unit norm,
zero mean, and the weight of 9 on the lowest b*m Ritz vectors.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2604_01800_gb300 import inputs as I  # noqa: E402
from paper_2604_01800_gb300 import train  # noqa: E402


class _OracleApply:
    """ppe_apply(grid, v, w) through the FP64 oracle's assembled operator."""

    def __init__(self, dx, dy):
        self.A = oracle.CSR(dx, dy)

    def ppe_apply(self, grid, v, w):
        w.copy_(torch.from_numpy(self.A.matvec(v.reshape(-1).numpy()).reshape(v.shape)))


class _Grid:
    def __init__(self, nx, ny):
        self.nx, self.ny = nx, ny


def _dct_eigenvalues(n):
    k = np.arange(n)
    s = np.sin(np.pi * k / (2 * n)) ** 2
    return np.unique(np.round(4.0 * (s[:, None] + s[None, :]).reshape(-1), 12))


@pytest.mark.parametrize("n", [8, 12])
def test_ritz_values_are_the_closed_form_spectrum(n):
    dx = dy = I.uniform_spacing(n)
    fake = _OracleApply(dx, dy)
    Q, theta = train.ritz_vectors(fake, _Grid(n, n), n * n, 3 * n * n // 2, seed=3, dev="cpu")
    lam = _dct_eigenvalues(n)
    lam = lam[lam > 1e-9]                                   # the constant null space is projected out
    # every Ritz value is an eigenvalue of A
    dist = np.min(np.abs(theta[:, None] - lam[None, :]), axis=1)
    assert np.all(dist <= 1e-9 * lam.max()), dist.max()
    # the extreme eigenvalues are found (a random start has weight on every eigenspace)
    assert abs(theta.min() - lam.min()) <= 1e-9 and abs(theta.max() - lam.max()) <= 1e-9 * lam.max()
    # and every eigenvalue of A in range(A) is among them (once the start
    # vector's Krylov space is exhausted, rounding seeds the remaining
    # directions, so degenerate eigenvalues may appear more than once)
    assert np.all(np.min(np.abs(lam[:, None] - theta[None, :]), axis=1) <= 1e-9 * lam.max())
    # Ritz vectors: orthonormal, zero mean, A q = theta q
    Qd = Q.double().numpy()
    assert np.allclose(Qd @ Qd.T, np.eye(len(theta)), atol=1e-5)
    assert np.allclose(Qd.sum(axis=1), 0.0, atol=1e-4)
    AQ = np.stack([fake.A.matvec(q) for q in Qd])
    assert np.allclose(AQ, theta[:, None] * Qd, atol=1e-4 * lam.max())


def test_few_lanczos_steps_find_the_extreme_eigenvalues():
    """m << N steps, as in the data recipe: the Ritz values lie inside
    [lambda_min, lambda_max] (Cauchy interlacing) and the extreme ones converge
    first (12 x 12 grid, 40 steps: both ends to 1e-6)."""
    n = 12
    dx = dy = I.uniform_spacing(n)
    lam = _dct_eigenvalues(n)
    lam = lam[lam > 1e-9]
    _, theta = train.ritz_vectors(_OracleApply(dx, dy), _Grid(n, n), n * n, 40, seed=3, dev="cpu")
    assert len(theta) == 40
    assert theta.min() >= lam.min() - 1e-12 and theta.max() <= lam.max() + 1e-12
    assert abs(theta.min() - lam.min()) <= 1e-6 and abs(theta.max() - lam.max()) <= 1e-6


def test_ritz_samples_follow_eqs_14_15():
    n, m, b = 12, 60, 0.6
    dx = dy = I.uniform_spacing(n)
    Q, theta = train.ritz_vectors(_OracleApply(dx, dy), _Grid(n, n), n * n, m, seed=5, dev="cpu")
    m = Q.shape[0]
    R = train.ritz_samples(Q, 400, b, I.rng(9))
    Rd = R.double().numpy()
    assert np.allclose(np.linalg.norm(Rd, axis=1), 1.0, atol=1e-5)           # Eq. 14: unit norm
    assert np.allclose(Rd.sum(axis=1), 0.0, atol=1e-4)                      # in range(A)
    # Eq. 15: c_j = 9 N(0,1) on the lowest b*m Ritz vectors, N(0,1) on the rest,
    # so the low block carries 81 b m / (81 b m + (1 - b) m) of the energy on average
    C = Rd @ Q.double().numpy().T
    low = int(b * m)
    share = (C[:, :low] ** 2).sum() / (C ** 2).sum()
    expect = 81 * low / (81 * low + (m - low))
    assert abs(share - expect) <= 0.01, (share, expect)
    assert np.all(np.diff(theta) >= 0)                                       # ordered by Ritz value
