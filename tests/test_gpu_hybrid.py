"""Hybrid (CG-type + DLSM) solves on the GPU, checked against the FP64 oracle.

The DLSM update (Eqs. 11-12) is validated with known directions before any
training: with the exact error A e = r_hat as the direction, the line search
takes alpha = 1 and removes the residual up to the FP32 rounding of e, so the
hybrid converges in a handful of iterations; with random directions it must
still reach the same solution (the exact line search never increases the
A-norm error); an untrained network likewise.  Every hybrid solve must reach
the same tolerance as plain PCG.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2604_01800_gb300 import inputs as I  # noqa: E402

pytestmark = pytest.mark.gpu
RES_TOL = 1e-8


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_01800_gb300 import api as A
    return A


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _check_solution(w, x, xo):
    xg = x.cpu().numpy()
    assert oracle.true_relres(w.dx, w.dy, w.f, xg) <= RES_TOL * 1.05
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-6


@pytest.fixture(scope="module")
def case():
    w = I.config1(2)
    xo, _, _ = oracle.solve(w.dx, w.dy, w.f, tol_rel=1e-11)
    return w, xo


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_exact_error_directions(api, case, prec):
    w, xo = case
    V = np.outer(w.dy, w.dx)
    calls = []

    def exact(r, e, stream):
        torch.cuda.synchronize()
        rh = r.double().cpu().numpy()
        rh = rh - rh.mean()
        # A e = rh with A = -V M  <=>  M e = -rh / V
        ee, _, st = oracle.solve(w.dx, w.dy, -rh / V, tol_rel=1e-12)
        calls.append(st)
        e.copy_(torch.tensor(ee, dtype=torch.float32, device="cuda"))
        torch.cuda.synchronize()

    grid = api.ppe_create_grid(w.dx, w.dy)
    api.ppe_set_direction_source(grid, exact)
    x = torch.zeros(w.ny, w.nx, dtype=torch.float64, device="cuda")
    p = api.PPE_PREC_MIXED if prec == "mixed" else api.PPE_PREC_FP64
    info = api.ppe_solve(grid, _dev(w.f), x, RES_TOL, api.PPE_MODE_HYBRID, p)
    assert info["iters_dlsm"] >= 1 and all(s == 0 for s in calls)
    assert info["iters_pcg"] + info["iters_dlsm"] <= 30, info
    _check_solution(w, x, xo)
    # plain PCG on the same system takes far longer
    x2 = torch.zeros_like(x)
    plain = api.ppe_solve(grid, _dev(w.f), x2, RES_TOL, api.PPE_MODE_PCG, p)
    assert plain["iters_pcg"] > 5 * (info["iters_pcg"] + info["iters_dlsm"])


def test_random_directions_still_converge(api, case):
    w, xo = case
    gen = torch.Generator(device="cuda").manual_seed(5)

    def noise(r, e, stream):
        e.copy_(torch.randn(e.shape, generator=gen, device="cuda"))

    grid = api.ppe_create_grid(w.dx, w.dy)
    api.ppe_set_direction_source(grid, noise)
    x = torch.zeros(w.ny, w.nx, dtype=torch.float64, device="cuda")
    info = api.ppe_solve(grid, _dev(w.f), x, RES_TOL, api.PPE_MODE_HYBRID, api.PPE_PREC_MIXED)
    assert info["status"] == 0 and info["net_calls"] >= 1
    _check_solution(w, x, xo)


def test_untrained_network_hybrid(api, case):
    w, xo = case
    net = api.net_create(api.net_default_config(), 3)
    grid = api.ppe_create_grid(w.dx, w.dy)
    net.attach(grid)
    x = torch.zeros(w.ny, w.nx, dtype=torch.float64, device="cuda")
    info = api.ppe_solve(grid, _dev(w.f), x, RES_TOL, api.PPE_MODE_HYBRID, api.PPE_PREC_MIXED, net=net)
    assert info["status"] == 0 and info["net_calls"] >= 1
    _check_solution(w, x, xo)


def test_hybrid_budget_falls_back_to_pcg(api, case):
    w, xo = case
    grid = api.ppe_create_grid(w.dx, w.dy)
    api.ppe_set_options(grid, hybrid_budget=7)

    def zero(r, e, stream):
        e.zero_()

    api.ppe_set_direction_source(grid, zero)
    x = torch.zeros(w.ny, w.nx, dtype=torch.float64, device="cuda")
    info = api.ppe_solve(grid, _dev(w.f), x, RES_TOL, api.PPE_MODE_HYBRID, api.PPE_PREC_MIXED)
    assert info["status"] == 0 and info["fell_back"] == 1
    assert info["dlsm_skipped"] >= 1          # a zero direction fails the curvature guard
    _check_solution(w, x, xo)


@pytest.mark.parametrize("limit", [6, 0])
def test_stall_limit_hands_useless_directions_to_pcg(api, case, limit):
    """A fixed random field as the direction barely moves the residual.  With
    dlsm_stall_limit = 6 the solve gives up on DLSM after such steps and
    finishes as plain PCG; with 0 it keeps alternating until the iteration
    budget.  Both reach the plain solution."""
    w, xo = case
    grid = api.ppe_create_grid(w.dx, w.dy)
    api.ppe_set_options(grid, dlsm_stall_limit=limit, hybrid_budget=60)
    gen = torch.Generator(device="cuda").manual_seed(7)
    fixed = torch.randn(w.ny, w.nx, generator=gen, device="cuda")

    def same(r, e, stream):
        e.copy_(fixed)

    api.ppe_set_direction_source(grid, same)
    x = torch.zeros(w.ny, w.nx, dtype=torch.float64, device="cuda")
    info = api.ppe_solve(grid, _dev(w.f), x, RES_TOL, api.PPE_MODE_HYBRID, api.PPE_PREC_MIXED)
    assert info["status"] == 0 and info["fell_back"] == 1
    if limit:
        assert limit <= info["iters_dlsm"] <= 2 * limit, info
    else:
        assert info["iters_dlsm"] >= 20, info            # 60 iterations of CG^3 DLSM^2 cycles
    _check_solution(w, x, xo)


def test_hybrid_without_source_is_an_error(api, case):
    w, _ = case
    grid = api.ppe_create_grid(w.dx, w.dy)
    x = torch.zeros(w.ny, w.nx, dtype=torch.float64, device="cuda")
    with pytest.raises(api.PPEError) as ei:
        api.ppe_solve(grid, _dev(w.f), x, RES_TOL, api.PPE_MODE_HYBRID, api.PPE_PREC_MIXED)
    assert ei.value.status == api._lib.PPE_ERR_NO_NET
