"""Parity of the CUDA solver path (through the C ABI) with the FP64 oracle.

Bars (from the hot-path target): true relative residual <= 1e-8 evaluated by
the oracle on the GPU's answer, and solution relative L2 error <= 1e-6
against the oracle's reference solution (solved to 1e-11), for both plain
FP64 PCG and mixed FP32/FP64 PCG.  The FP64 operator is compared entry by
entry: both sides evaluate the same five products per row, so only the
summation order differs (bound 1e-13 relative to the row scale).
"""
import functools

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2604_01800_gb300 import inputs as I  # noqa: E402

pytestmark = pytest.mark.gpu

SOL_TOL = 1e-6
RES_TOL = 1e-8


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_01800_gb300 import api as A
    return A


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@functools.lru_cache(maxsize=None)
def _ref(key):
    w = _WORK[key]()
    x, info, st = oracle.solve(w.dx, w.dy, w.f, tol_rel=1e-11)
    return w, x


def _ragged(nx, ny, seed):
    g = I.rng(seed)
    dx, dy = I.random_spacing(nx, g), I.random_spacing(ny, g)
    return I.Workload(f"ragged{nx}x{ny}", dx, dy, I.gaussian_rhs(dx, dy, g, 6))


_WORK = {
    "c1": lambda: I.config1(0),
    "c1b": lambda: I.config1(1),
    "c2": lambda: I.config2(0),
    "c3": lambda: I.config3(0),
    "r37x300": lambda: _ragged(37, 300, 5),
    "r129x131": lambda: _ragged(129, 131, 6),
    "r5x7": lambda: _ragged(5, 7, 7),
    "r1x50": lambda: _ragged(1, 50, 8),
    "r260x9": lambda: _ragged(260, 9, 9),
}


@pytest.mark.parametrize("nx,ny,seed", [(5, 7, 1), (33, 17, 2), (130, 9, 3), (200, 150, 4), (1, 1, 5), (1, 40, 6)])
def test_apply_matches_oracle(api, nx, ny, seed):
    g0 = I.rng(seed)
    dx, dy = g0.uniform(0.1, 2.0, nx), g0.uniform(0.1, 2.0, ny)
    x = g0.standard_normal((ny, nx))
    grid = api.ppe_create_grid(dx, dy)
    y = torch.zeros(ny, nx, dtype=torch.float64, device="cuda")
    api.ppe_apply(grid, _dev(x), y)
    torch.cuda.synchronize()
    yo = oracle.apply(dx, dy, x)
    A = oracle.CSR(dx, dy)
    rowscale = np.abs(A.scipy()).dot(np.abs(x).reshape(-1)).reshape(ny, nx) + 1e-300
    assert np.max(np.abs(y.cpu().numpy() - yo) / rowscale) <= 1e-13


def _check(api, key, prec, x0=None, **opts):
    w, xo = _ref(key)
    grid = api.ppe_create_grid(w.dx, w.dy, w.mask)
    if opts:
        api.ppe_set_options(grid, **opts)
    rhs = _dev(w.f)
    x = _dev(x0) if x0 is not None else torch.zeros_like(rhs)
    info = api.ppe_solve(grid, rhs, x, RES_TOL, api.PPE_MODE_PCG, prec)
    xg = x.cpu().numpy()
    rr = oracle.true_relres(w.dx, w.dy, w.f, xg)
    err = np.linalg.norm(xg - xo) / np.linalg.norm(xo)
    V = np.outer(w.dy, w.dx)
    assert info["status"] == 0, info
    assert rr <= RES_TOL * 1.05, (rr, info)
    assert err <= SOL_TOL, (err, info)
    assert abs((V * xg).sum()) <= 1e-12 * np.abs(V * xg).sum() + 1e-300
    # the device's own FP64 residual report agrees with the oracle's evaluation
    # (below ~1e-11 both evaluations are dominated by FP64 rounding of b - A x)
    assert abs(info["rel_res_true"] - rr) <= 1e-3 * rr + 1e-11
    return info


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("key", ["c1", "r37x300", "r129x131", "r5x7", "r1x50", "r260x9"])
def test_solve_small(api, key, prec):
    _check(api, key, api.PPE_PREC_FP64 if prec == "fp64" else api.PPE_PREC_MIXED)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_solve_config2_512(api, prec):
    info = _check(api, "c2", api.PPE_PREC_FP64 if prec == "fp64" else api.PPE_PREC_MIXED)
    if prec == "mixed":
        assert info["refinements"] >= 2


def test_solve_config3_cylinder_mask(api):
    _check(api, "c3", api.PPE_PREC_MIXED)


def test_warm_start(api):
    w, xo = _ref("c1b")
    x0 = xo + 0.01 * I.rng(3).standard_normal(xo.shape)
    info = _check(api, "c1b", api.PPE_PREC_MIXED, x0=x0)
    cold = _check(api, "c1b", api.PPE_PREC_MIXED)
    assert info["iters_pcg"] < cold["iters_pcg"]


def test_incompatible_rhs(api):
    w = I.config1(0)
    grid = api.ppe_create_grid(w.dx, w.dy)
    x = torch.zeros(w.ny, w.nx, dtype=torch.float64, device="cuda")
    info = api.ppe_solve(grid, _dev(w.f + 1.0), x, 1e-8, api.PPE_MODE_PCG, api.PPE_PREC_MIXED,
                         raise_on_error=False)
    assert info["status"] == api._lib.PPE_ERR_INCOMPATIBLE_RHS
    assert info["incompat"] > 1e-6


def test_zero_rhs(api):
    w = I.config1(0)
    grid = api.ppe_create_grid(w.dx, w.dy)
    x = torch.ones(w.ny, w.nx, dtype=torch.float64, device="cuda")
    info = api.ppe_solve(grid, torch.zeros_like(x), x, 1e-8, api.PPE_MODE_PCG, api.PPE_PREC_MIXED)
    assert info["status"] == 0 and float(x.abs().max()) == 0.0


def test_iteration_cap_reports_not_converged(api):
    w = I.config1(0)
    grid = api.ppe_create_grid(w.dx, w.dy)
    api.ppe_set_options(grid, max_iters=5)
    x = torch.zeros(w.ny, w.nx, dtype=torch.float64, device="cuda")
    info = api.ppe_solve(grid, _dev(w.f), x, 1e-8, api.PPE_MODE_PCG, api.PPE_PREC_MIXED, raise_on_error=False)
    assert info["status"] == api._lib.PPE_ERR_NOT_CONVERGED
    assert np.all(np.isfinite(x.cpu().numpy()))


def test_batch_matches_single(api):
    keys = ["c1", "r37x300", "r129x131", "r5x7", "r260x9"]
    grids, rhs, xs, refs = [], [], [], []
    for k in keys:
        w, xo = _ref(k)
        grids.append(api.ppe_create_grid(w.dx, w.dy))
        rhs.append(_dev(w.f))
        xs.append(torch.zeros_like(rhs[-1]))
        refs.append((w, xo))
    infos, st = api.ppe_solve_batch(grids, rhs, xs, RES_TOL, api.PPE_MODE_PCG, api.PPE_PREC_MIXED)
    assert st == 0
    for (w, xo), x, info in zip(refs, xs, infos):
        xg = x.cpu().numpy()
        assert info["status"] == 0
        assert oracle.true_relres(w.dx, w.dy, w.f, xg) <= RES_TOL * 1.05
        assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= SOL_TOL


def test_repeatable_bitwise(api):
    w, _ = _ref("r129x131")
    grid = api.ppe_create_grid(w.dx, w.dy)
    outs = []
    for _ in range(2):
        x = torch.zeros(w.ny, w.nx, dtype=torch.float64, device="cuda")
        api.ppe_solve(grid, _dev(w.f), x, RES_TOL, api.PPE_MODE_PCG, api.PPE_PREC_MIXED)
        outs.append(x.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("iter_pass", [1, 2])
@pytest.mark.parametrize("key", ["c1", "r37x300", "r129x131", "r260x9", "r1x50"])
def test_iteration_pass_variants(api, key, iter_pass):
    """The tile-cooperative (1) and streaming (2) FP32 iteration passes both
    meet the parity bars on ragged grids."""
    _check(api, key, api.PPE_PREC_MIXED, iter_pass=iter_pass)


def test_streaming_pass_runs_across_tile_columns(api):
    """620 x 1000 cells: 5 tile columns of 63 tiles over at most one block per
    SM, so the tile runs of some warps end in one column and continue in the
    next.  Both passes reach the tolerance (checked by the oracle) and agree."""
    g = I.rng(77)
    dx, dy = I.random_spacing(620, g), I.random_spacing(1000, g)
    f = I.gaussian_rhs(dx, dy, g, 6)
    grid = api.ppe_create_grid(dx, dy)
    xs = []
    for iter_pass in (1, 2):
        api.ppe_set_options(grid, iter_pass=iter_pass)
        x = torch.zeros(len(dy), len(dx), dtype=torch.float64, device="cuda")
        info = api.ppe_solve(grid, _dev(f), x, RES_TOL, api.PPE_MODE_PCG, api.PPE_PREC_MIXED)
        assert info["status"] == 0
        xg = x.cpu().numpy()
        assert oracle.true_relres(dx, dy, f, xg) <= RES_TOL * 1.05
        xs.append(xg)
    assert np.linalg.norm(xs[0] - xs[1]) <= 1e-6 * np.linalg.norm(xs[0])


def test_batch_streaming_pass(api):
    keys = ["c1", "r37x300", "r129x131", "r260x9"]
    grids, rhs, xs, refs = [], [], [], []
    for k in keys:
        w, xo = _ref(k)
        grids.append(api.ppe_create_grid(w.dx, w.dy))
        api.ppe_set_options(grids[-1], iter_pass=2)
        rhs.append(_dev(w.f))
        xs.append(torch.zeros_like(rhs[-1]))
        refs.append((w, xo))
    infos, st = api.ppe_solve_batch(grids, rhs, xs, RES_TOL, api.PPE_MODE_PCG, api.PPE_PREC_MIXED)
    assert st == 0
    for (w, xo), x, info in zip(refs, xs, infos):
        xg = x.cpu().numpy()
        assert info["status"] == 0
        assert oracle.true_relres(w.dx, w.dy, w.f, xg) <= RES_TOL * 1.05
        assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= SOL_TOL


@pytest.mark.parametrize("prec", ["mixed", "fp64", "multigrid"])
def test_solution_scales_exactly_with_the_source(api, prec):
    """Cross-block sums are float-float (FP32's exponent range) and the inner
    vectors of the mixed and multigrid solves are FP32, so the solver works on
    the system scaled by a power of two (the binary exponent of max |b|, or of
    the residual norm for an inner solve); the scaling is exact.  A source
    multiplied by 2^k must give the solution multiplied by 2^k bit for bit,
    for k = +-110, where |b|^2 lies far outside FP32's range."""
    w = I.config1(0)
    grid = api.ppe_create_grid(w.dx, w.dy)
    if prec == "multigrid":
        api.ppe_set_options(grid, preconditioner=1)
    p = api.PPE_PREC_FP64 if prec == "fp64" else api.PPE_PREC_MIXED
    out = {}
    for k in (0, -110, 110):
        x = torch.zeros(w.ny, w.nx, dtype=torch.float64, device="cuda")
        info = api.ppe_solve(grid, _dev(np.ldexp(w.f, k)), x, 1e-8, api.PPE_MODE_PCG, p)
        assert info["status"] == 0 and info["rel_res_true"] <= 1e-8, (k, info)
        out[k] = (x.cpu().numpy(), info["iters_pcg"])
    x0, it0 = out[0]
    assert np.abs(x0).max() > 0
    for k in (-110, 110):
        xk, itk = out[k]
        assert itk == it0, (k, itk, it0)
        assert np.array_equal(np.ldexp(xk, -k), x0), k
    grid.close()


@pytest.mark.parametrize("tile_rows", [4, 8, 16])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("key", ["c1", "r37x300", "r129x131", "r5x7", "r260x9"])
def test_tile_heights(api, key, prec, tile_rows):
    """Every tile height of the tile-cooperative kernels (16 rows; 8 or 4
    rows, which small grids take by default to spread over more blocks)
    meets the parity bars on ragged grids.  r37x300 has 19, 38 or 75 tiles
    (300 rows end in a tail of 12, 4 or a whole tile), so several blocks
    share the system; r5x7 fits in part of one tile."""
    _check(api, key, api.PPE_PREC_FP64 if prec == "fp64" else api.PPE_PREC_MIXED, tile_rows=tile_rows)


@pytest.mark.parametrize("tile_rows", [4, 8])
def test_tile_heights_c3(api, tile_rows):
    """The 256x256 cylinder grid (128 or 64 tiles, one per block) with a
    short tile height reaches the same answer as with 16 rows: iteration counts within a few and
    solutions within the solution bar of each other and of the oracle."""
    info = _check(api, "c3", api.PPE_PREC_MIXED, tile_rows=tile_rows)
    ref = _check(api, "c3", api.PPE_PREC_MIXED, tile_rows=16)
    assert abs(info["iters_pcg"] - ref["iters_pcg"]) <= 0.02 * ref["iters_pcg"] + 5, (info, ref)


@pytest.mark.parametrize("tile_rows", [4, 8])
def test_batch_short_tiles(api, tile_rows):
    """A batch of small systems on short tiles: every system meets the
    parity bars."""
    keys = ["c1", "r37x300", "r129x131", "r260x9"]
    grids, rhs, xs, refs = [], [], [], []
    for k in keys:
        w, xo = _ref(k)
        grids.append(api.ppe_create_grid(w.dx, w.dy))
        api.ppe_set_options(grids[-1], tile_rows=tile_rows)
        rhs.append(_dev(w.f))
        xs.append(torch.zeros_like(rhs[-1]))
        refs.append((w, xo))
    infos, st = api.ppe_solve_batch(grids, rhs, xs, RES_TOL, api.PPE_MODE_PCG, api.PPE_PREC_MIXED)
    assert st == 0
    for (w, xo), x, info in zip(refs, xs, infos):
        xg = x.cpu().numpy()
        assert info["status"] == 0
        assert oracle.true_relres(w.dx, w.dy, w.f, xg) <= RES_TOL * 1.05
        assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= SOL_TOL
