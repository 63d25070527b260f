"""Failure paths, made to happen without faulting the GPU.

* Bounded barrier wait: a test hook makes one block of the persistent solver
  kernel withhold its partial sums once.  The other blocks' waits (bounded
  by spin_limit_ms) expire; every block returns, and the solve reports
  PPE_ERR_TIMEOUT, in both drivers.  The grid then solves normally.
* Non-finite input: a NaN in the initial guess makes the FP64 true residual
  non-finite, which ends the solve with PPE_ERR_NAN.
* Non-finite DLSM direction: the curvature guard (e.Ae compared with
  guard * e.e * max diag) rejects it; the solve goes on with CG and reaches
  the oracle's solution.
* Stalled FP32 inner iteration: a test hook makes the mixed solve's stall
  rule fire; the solve continues in FP64 from its iterate, in both drivers.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2604_01800_gb300 import inputs as I  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-8


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_01800_gb300 import api as A
    return A


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("host_loop", [0, 1])
@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_withheld_record_times_out(api, host_loop, prec):
    w = I.config3(0)                               # 256^2: 32 tiles, so several blocks share the system
    p = api.PPE_PREC_MIXED if prec == "mixed" else api.PPE_PREC_FP64
    grid = api.ppe_create_grid(w.dx, w.dy)
    api.ppe_set_options(grid, debug_skip_block=2, spin_limit_ms=20, host_loop=host_loop)
    x = torch.zeros(w.ny, w.nx, dtype=torch.float64, device="cuda")
    info = api.ppe_solve(grid, _dev(w.f), x, TOL, api.PPE_MODE_PCG, p, raise_on_error=False)
    assert info["status"] == api._lib.PPE_ERR_TIMEOUT, info
    assert b"wait expired" in api._lib.load().ppe_last_error()
    torch.cuda.synchronize()                       # the context is intact
    api.ppe_set_options(grid, host_loop=host_loop)
    info = api.ppe_solve(grid, _dev(w.f), x, TOL, api.PPE_MODE_PCG, p)
    assert info["status"] == 0
    assert oracle.true_relres(w.dx, w.dy, w.f, x.cpu().numpy()) <= TOL * 1.05


def test_nan_initial_guess_reports_nan(api):
    w = I.config1(1)
    grid = api.ppe_create_grid(w.dx, w.dy)
    x = torch.zeros(w.ny, w.nx, dtype=torch.float64, device="cuda")
    x[5, 7] = float("nan")
    info = api.ppe_solve(grid, _dev(w.f), x, TOL, api.PPE_MODE_PCG, api.PPE_PREC_MIXED, raise_on_error=False)
    assert info["status"] == api._lib.PPE_ERR_NAN, info
    x.zero_()
    assert api.ppe_solve(grid, _dev(w.f), x, TOL, api.PPE_MODE_PCG, api.PPE_PREC_MIXED)["status"] == 0


def test_nan_direction_is_rejected(api):
    w = I.config1(2)
    xo, _, _ = oracle.solve(w.dx, w.dy, w.f, tol_rel=1e-11)
    grid = api.ppe_create_grid(w.dx, w.dy)
    api.ppe_set_options(grid, hybrid_budget=40)

    def nan_source(r, e, stream):
        e.fill_(float("nan"))

    api.ppe_set_direction_source(grid, nan_source)
    x = torch.zeros(w.ny, w.nx, dtype=torch.float64, device="cuda")
    info = api.ppe_solve(grid, _dev(w.f), x, TOL, api.PPE_MODE_HYBRID, api.PPE_PREC_MIXED)
    assert info["status"] == 0 and info["dlsm_skipped"] >= 1 and info["iters_dlsm"] == 0, info
    xg = x.cpu().numpy()
    assert oracle.true_relres(w.dx, w.dy, w.f, xg) <= TOL * 1.05
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-6


@pytest.mark.parametrize("shape", [(4096, 16), (16, 4096)])
def test_ill_conditioned_strip_mixed_solve_converges(api, shape):
    """A long strip: the FP64 Jacobi-PCG needs ~30,000 iterations, and the
    condition number is near the reciprocal of FP32's precision, so an FP32
    inner solve loses its reduction target: its recursive residual stops
    tracking the true one.  The inner solve's length budget (2000 + 4x the
    last successful one) then forces residual replacements often enough for
    the mixed solve to keep converging (measured: 2-3x FP64's iteration
    count at a fifth to a tenth of its cost per iteration); should the true
    residual stop halving for three refinements, the solve continues in
    FP64 instead.  Either way it must reach the tolerance."""
    g = I.rng(43)
    nx, ny = shape
    dx, dy = I.random_spacing(nx, g), I.random_spacing(ny, g)
    f = I.gaussian_rhs(dx, dy, g, 6)
    grid = api.ppe_create_grid(dx, dy)
    x = torch.zeros(ny, nx, dtype=torch.float64, device="cuda")
    info = api.ppe_solve(grid, _dev(f), x, TOL, api.PPE_MODE_PCG, api.PPE_PREC_MIXED)
    assert info["status"] == 0, info
    assert info["iters_pcg"] <= 150_000, info
    assert oracle.true_relres(dx, dy, f, x.cpu().numpy()) <= TOL * 1.05


@pytest.mark.parametrize("host_loop", [0, 1])
def test_stalled_mixed_solve_continues_in_fp64(api, host_loop):
    """The FP64 continuation: a test hook makes the mixed solve count every
    refinement after the first as one that failed to halve the true residual
    (no real system has been found on which FP32 inner iterations stall), so
    the stall rule ends the FP32 iteration after three of them; the solve
    then continues in FP64 from its iterate and reaches the oracle's
    solution, with both phases' iterations in the report."""
    w = I.config3(0)
    grid = api.ppe_create_grid(w.dx, w.dy)
    api.ppe_set_options(grid, debug_force_stall=1, host_loop=host_loop)
    x = torch.zeros(w.ny, w.nx, dtype=torch.float64, device="cuda")
    info = api.ppe_solve(grid, _dev(w.f), x, TOL, api.PPE_MODE_PCG, api.PPE_PREC_MIXED)
    assert info["status"] == 0 and info["precision_fallback"] == 1, info
    assert info["refinements"] >= 4, info
    xg = x.cpu().numpy()
    assert oracle.true_relres(w.dx, w.dy, w.f, xg) <= TOL * 1.05
    xo, _, _ = oracle.solve(w.dx, w.dy, w.f, tol_rel=1e-11)
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-6
    grid.close()


def test_well_conditioned_mixed_solve_stays_mixed(api):
    w = I.config2(0)
    grid = api.ppe_create_grid(w.dx, w.dy)
    x = torch.zeros(w.ny, w.nx, dtype=torch.float64, device="cuda")
    info = api.ppe_solve(grid, _dev(w.f), x, TOL, api.PPE_MODE_PCG, api.PPE_PREC_MIXED)
    assert info["status"] == 0 and info["precision_fallback"] == 0, info
