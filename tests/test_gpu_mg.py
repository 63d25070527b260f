"""The multigrid partner (ppe_solve_opts.preconditioner = 1) against the oracle.

* One V-cycle, element by element, against oracle/mg.py's FP64 V-cycle on the
  same residual: the GPU evaluates it in FP32 (line solves by the Thomas
  algorithm with FP32 factors), so the bar is a relative L2 difference of
  1e-4, about 1000 FP32 roundings.  Grids cover a hierarchy run entirely
  inside one block, one with grid-wide levels above it, odd sizes on every
  level, and a long strip whose short axis stops coarsening at one cell.
* Whole solves: the true relative residual (evaluated by the oracle in FP64)
  within the tolerance, the solution within 1e-6 of the plain oracle's, zero
  volume-weighted mean, and an iteration count close to the FP64 oracle
  MG-PCG's (the FP32 inner iterations and the refinement restarts cost a
  few more).
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import mg  # noqa: E402
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


def _ragged(nx, ny, seed):
    g = I.rng(seed)
    dx, dy = I.random_spacing(nx, g), I.random_spacing(ny, g)
    return dx, dy, I.gaussian_rhs(dx, dy, g, 6)


@pytest.mark.parametrize("shape", [(13, 10), (64, 64), (300, 200), (521, 131), (2048, 9)])
def test_vcycle_matches_oracle(api, shape):
    nx, ny = shape
    dx, dy, _ = _ragged(nx, ny, 60 + nx)
    grid = api.ppe_create_grid(dx, dy)
    r = I.rng(nx + ny).standard_normal(nx * ny)
    r -= r.mean()
    rt = torch.tensor(r.reshape(ny, nx), dtype=torch.float32, device="cuda")
    zt = torch.zeros_like(rt)
    L = api._lib.load()
    st = L.ppe_debug_mg_vcycle(grid.handle, ctypes.c_void_p(rt.data_ptr()), ctypes.c_void_p(zt.data_ptr()),
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    api._lib.check(st, "ppe_debug_mg_vcycle")
    M = mg.MGPreconditioner(dx, dy)
    zo = M(rt.double().cpu().numpy().reshape(-1))
    zg = zt.double().cpu().numpy().reshape(-1)
    rel = np.linalg.norm(zg - zo) / np.linalg.norm(zo)
    assert rel <= 1e-4, rel


@pytest.mark.parametrize("case", ["c1", "c3", "c2", "ragged"])
def test_mgpcg_solve_matches_oracle(api, case):
    if case == "ragged":
        dx, dy, f = _ragged(333, 141, 9)
    else:
        w = {"c1": I.config1(0), "c2": I.config2(0), "c3": I.config3(0)}[case]
        dx, dy, f = w.dx, w.dy, w.f
    grid = api.ppe_create_grid(dx, dy)
    api.ppe_set_options(grid, preconditioner=1)
    x = torch.zeros(dy.size, dx.size, dtype=torch.float64, device="cuda")
    info = api.ppe_solve(grid, _dev(f), x, TOL, api.PPE_MODE_PCG, api.PPE_PREC_MIXED)
    xg = x.cpu().numpy()
    assert info["status"] == 0
    assert oracle.true_relres(dx, dy, f, xg) <= TOL * 1.05
    xo, _, _ = oracle.solve(dx, dy, f, tol_rel=1e-11)
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-6
    V = np.outer(dy, dx)
    assert abs((V * xg).sum()) <= 1e-10 * (V * np.abs(xg)).sum()
    _, oi = mg.mgpcg_solve(dx, dy, f, tol_rel=TOL)
    assert info["iters_pcg"] <= 2 * oi["iters"] + 6, (info["iters_pcg"], oi["iters"])


def test_mgpcg_full_size_sequence_grid(api):
    """The 2048 x 1024 wake-refined grid (spacing ratio 123), two warm-started
    steps, checked by the oracle's true residual and the zero mean."""
    dx, dy, bodies = I.config5_grid()
    grid = api.ppe_create_grid(dx, dy)
    api.ppe_set_options(grid, preconditioner=1)
    x = torch.zeros(dy.size, dx.size, dtype=torch.float64, device="cuda")
    for t in range(2):
        f = I.config5_rhs(t, dx, dy, bodies)
        info = api.ppe_solve(grid, _dev(f), x, TOL, api.PPE_MODE_PCG, api.PPE_PREC_MIXED)
        assert info["status"] == 0 and info["iters_pcg"] <= 60, info
        xg = x.cpu().numpy()
        assert oracle.true_relres(dx, dy, f, xg) <= TOL * 1.05
        V = np.outer(dy, dx)
        assert abs((V * xg).sum()) <= 1e-10 * (V * np.abs(xg)).sum()


@pytest.mark.parametrize("shape", [(4096, 16), (16, 4096)])
def test_mgpcg_long_strips(api, shape):
    """The strips on which FP32 Jacobi-PCG stalls: the line smoother along the
    long axis resolves them in a few iterations."""
    dx, dy, f = _ragged(*shape, 43)
    grid = api.ppe_create_grid(dx, dy)
    api.ppe_set_options(grid, preconditioner=1)
    x = torch.zeros(shape[1], shape[0], dtype=torch.float64, device="cuda")
    info = api.ppe_solve(grid, _dev(f), x, TOL, api.PPE_MODE_PCG, api.PPE_PREC_MIXED)
    assert info["status"] == 0 and info["iters_pcg"] <= 60, info
    assert oracle.true_relres(dx, dy, f, x.cpu().numpy()) <= TOL * 1.05


def test_mgpcg_refuses_what_it_does_not_run(api):
    w = I.config1(0)
    grid = api.ppe_create_grid(w.dx, w.dy)
    api.ppe_set_options(grid, preconditioner=1)
    x = torch.zeros(w.ny, w.nx, dtype=torch.float64, device="cuda")
    for mode, prec in ((api.PPE_MODE_PCG, api.PPE_PREC_FP64), (api.PPE_MODE_HYBRID, api.PPE_PREC_MIXED)):
        with pytest.raises(api.PPEError) as ei:
            api.ppe_solve(grid, _dev(w.f), x, TOL, mode, prec, net=None)
        assert ei.value.status in (api._lib.PPE_ERR_ARG, api._lib.PPE_ERR_NO_NET)
    infos, st = api.ppe_solve_batch([grid], [_dev(w.f)], [x], TOL, api.PPE_MODE_PCG, api.PPE_PREC_MIXED,
                                    raise_on_error=False)
    assert st == api._lib.PPE_ERR_ARG
