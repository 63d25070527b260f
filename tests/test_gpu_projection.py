"""The projection kernels (Sec. 2.1 Eqs. 6-8) against oracle/projection.py,
and one whole projection step: source, PPE solve, correction, after which the
discrete divergence (evaluated by the oracle in FP64) vanishes to the solve's
tolerance."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import projection as PJ  # noqa: E402
from paper_2604_01800_gb300 import inputs as I  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_01800_gb300 import api as A
    return A


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _fields(nx, ny, seed):
    g = I.rng(seed)
    dx, dy = I.random_spacing(nx, g), I.random_spacing(ny, g)
    u = g.standard_normal((ny, nx + 1))
    v = g.standard_normal((ny + 1, nx))
    return dx, dy, u, v, g


@pytest.mark.parametrize("shape", [(7, 5), (130, 67), (512, 256)])
def test_source_and_correction_match_oracle(api, shape):
    nx, ny = shape
    dx, dy, u, v, g = _fields(nx, ny, nx)
    dt = 0.013
    grid = api.ppe_create_grid(dx, dy)
    S = torch.empty(ny, nx, dtype=torch.float64, device="cuda")
    api.ppe_source(grid, _dev(u), _dev(v), dt, S)
    So = PJ.ppe_source(dx, dy, u, v, dt)
    assert np.allclose(S.cpu().numpy(), So, rtol=1e-13, atol=1e-13 * np.abs(So).max())
    dp = g.standard_normal((ny, nx))
    p = g.standard_normal((ny, nx))
    du, dv, dpp = _dev(u), _dev(v), _dev(p)
    api.ppe_project(grid, _dev(dp), dt, du, dv, dpp)
    uo, vo, po = PJ.project(dx, dy, u, v, p, dp, dt)
    for a, b in ((du, uo), (dv, vo), (dpp, po)):
        assert np.allclose(a.cpu().numpy(), b, rtol=1e-13, atol=1e-13 * np.abs(b).max())


@pytest.mark.parametrize("precond", [0, 1])
def test_projection_step_removes_the_divergence(api, precond):
    """u* with walls at rest on the 256^2 cylinder grid: after S, the PPE
    solve (Jacobi or multigrid partner) and the correction, max |D u| is
    below 1e-6 of max |D u*|."""
    w = I.config3(0)
    dx, dy = w.dx, w.dy
    g = I.rng(77)
    u = g.standard_normal((dy.size, dx.size + 1))
    v = g.standard_normal((dy.size + 1, dx.size))
    u[:, [0, -1]] = 0.0
    v[[0, -1], :] = 0.0
    dt = 0.01
    grid = api.ppe_create_grid(dx, dy)
    api.ppe_set_options(grid, preconditioner=precond)
    du, dv = _dev(u), _dev(v)
    S = torch.empty(dy.size, dx.size, dtype=torch.float64, device="cuda")
    api.ppe_source(grid, du, dv, dt, S)
    dp = torch.zeros_like(S)
    info = api.ppe_solve(grid, S, dp, 1e-10, api.PPE_MODE_PCG, api.PPE_PREC_MIXED)
    assert info["status"] == 0
    api.ppe_project(grid, dp, dt, du, dv)
    div = PJ.divergence(dx, dy, du.cpu().numpy(), dv.cpu().numpy())
    assert np.abs(div).max() <= 1e-6 * np.abs(PJ.divergence(dx, dy, u, v)).max()
