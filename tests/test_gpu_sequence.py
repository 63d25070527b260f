"""Time sequence of PPE solves with warm starts (the projection loop's use of
the solver: one solve per time step, initial guess = previous pressure
increment), on a reduced version of the wake-refined cylinder grid.  Every
step must match the FP64 oracle; warm starts must not cost more iterations
than cold starts."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2604_01800_gb300 import inputs as I  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_01800_gb300 import api as A
    return A


def test_warm_started_sequence(api):
    dx, dy, bodies = I.config5_grid(256, 128)
    grid = api.ppe_create_grid(dx, dy)
    x = torch.zeros(dy.size, dx.size, dtype=torch.float64, device="cuda")
    warm, cold = [], []
    for t in range(4):
        f = I.config5_rhs(t, dx, dy, bodies)
        rhs = torch.tensor(f, dtype=torch.float64, device="cuda")
        info = api.ppe_solve(grid, rhs, x, 1e-8, api.PPE_MODE_PCG, api.PPE_PREC_MIXED)   # warm: x from step t-1
        xo, _, _ = oracle.solve(dx, dy, f, tol_rel=1e-11)
        xg = x.cpu().numpy()
        assert oracle.true_relres(dx, dy, f, xg) <= 1.05e-8
        assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-6
        xc = torch.zeros_like(x)
        cinfo = api.ppe_solve(grid, rhs, xc, 1e-8, api.PPE_MODE_PCG, api.PPE_PREC_MIXED)
        warm.append(info["iters_pcg"])
        cold.append(cinfo["iters_pcg"])
    assert sum(warm[1:]) <= sum(cold[1:])
