"""Parity of the GPU hybrid solve with the FP64 oracle's HyDEA solve.

Both sides get the same deterministic direction map (a blend of the exact
pseudo-inverse and the Jacobi inverse, a stand-in for a trained network that
helps but is not exact), so the alternation of CG phases and DLSM steps, the
step lengths and the convergence test are compared on the same sequence.
The grid spans two tiles in each direction with ragged tails.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import hybrid as H  # noqa: E402
from paper_2604_01800_gb300 import inputs as I  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_01800_gb300 import api as A
    return A


def _pinv(A):
    w, Q = np.linalg.eigh(A)
    keep = w > 1e-10 * w.max()
    return (Q[:, keep] / w[keep]) @ Q[:, keep].T


@pytest.fixture(scope="module")
def case():
    g = I.rng(4242)
    nx, ny = 136, 20
    dx = I.random_spacing(nx, g)
    dy = I.random_spacing(ny, g)
    S = I.gaussian_rhs(dx, dy, g)
    A = oracle.CSR(dx, dy).dense()
    return dx, dy, S, _pinv(A), np.diag(1.0 / np.diag(A))


@pytest.mark.parametrize("theta", [0.0, 0.2, 0.4])
@pytest.mark.parametrize("num_cg,num_dlsm", [(3, 2), (2, 1)])
def test_fp64_hybrid_follows_the_oracle(api, case, num_cg, num_dlsm, theta):
    dx, dy, S, P, Dinv = case
    M = (1 - theta) * P + theta * Dinv
    ny, nx = S.shape
    # the direction interface is FP32 (the network's): both sides get r_hat and
    # return e rounded to FP32
    f32 = lambda v: v.astype(np.float32).astype(np.float64)
    xo, io = H.hybrid_solve(dx, dy, S, lambda rh: f32((M @ f32(rh).reshape(-1)).reshape(ny, nx)), tol_rel=1e-8,
                            num_cg=num_cg, num_dlsm=num_dlsm)
    assert io["rel_res_true"] <= 1e-8 and io["fell_back"] == 0 and io["iters_dlsm"] >= 1
    Mg = torch.tensor(M, dtype=torch.float64, device="cuda")

    def direction(r, e, stream):
        e.copy_((Mg @ r.double().reshape(-1)).reshape(ny, nx).float())

    grid = api.ppe_create_grid(dx, dy)
    api.ppe_set_options(grid, num_cg=num_cg, num_dlsm=num_dlsm, dlsm_stall_limit=0)   # the oracle has no give-up rule
    api.ppe_set_direction_source(grid, direction)
    x = torch.zeros(ny, nx, dtype=torch.float64, device="cuda")
    info = api.ppe_solve(grid, torch.tensor(S, device="cuda"), x, 1e-8, api.PPE_MODE_HYBRID, api.PPE_PREC_FP64)
    assert info["status"] == 0 and info["rel_res_true"] <= 1e-8 and info["fell_back"] == 0
    # same alternation: the iteration counts of both kinds agree (one iteration of
    # slack: the device stops at 0.9 tol on its recursive residual before
    # confirming with the true one, the oracle at tol)
    assert abs(info["iters_pcg"] - io["iters_pcg"]) <= 1, (info, io["iters_pcg"], io["iters_dlsm"])
    assert abs(info["iters_dlsm"] - io["iters_dlsm"]) <= 1, (info, io["iters_pcg"], io["iters_dlsm"])
    xg = x.cpu().numpy()
    assert np.linalg.norm(xg - xo) <= 1e-6 * np.linalg.norm(xo)


def test_mixed_hybrid_reaches_the_oracle_solution(api, case):
    dx, dy, S, P, Dinv = case
    M = 0.6 * P + 0.4 * Dinv
    ny, nx = S.shape
    xr, _, _ = oracle.solve(dx, dy, S, tol_rel=1e-11)
    Mg = torch.tensor(M, dtype=torch.float64, device="cuda")

    def direction(r, e, stream):
        e.copy_((Mg @ r.double().reshape(-1)).reshape(ny, nx).float())

    grid = api.ppe_create_grid(dx, dy)
    api.ppe_set_direction_source(grid, direction)
    x = torch.zeros(ny, nx, dtype=torch.float64, device="cuda")
    info = api.ppe_solve(grid, torch.tensor(S, device="cuda"), x, 1e-8, api.PPE_MODE_HYBRID, api.PPE_PREC_MIXED)
    assert info["status"] == 0 and info["rel_res_true"] <= 1e-8 and info["iters_dlsm"] >= 2
    assert oracle.true_relres(dx, dy, S, x.cpu().numpy()) <= 1.05e-8
    assert np.linalg.norm(x.cpu().numpy() - xr) <= 1e-6 * np.linalg.norm(xr)
