"""The allocation-free solve entry point against the regular one.

ppe_solve_noalloc exists for callers that cannot allocate device memory (a
host whose device memory is reserved up front by its own pool allocator, a
loop that must not allocate after initialisation, a plugin whose host forbids
device allocations).  It takes its scratch from a fixed array inside the
library.  These checks call it through the C ABI twice in a row, on two
different systems, and compare each answer with ppe_solve's on the same
system, to the solution tolerance the other solver tests use; they also
check that an oversized grid is refused with a clear message.  This file
sorts last so that a run stopping at the first failure has run every other
test before it.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2604_01800_gb300 import inputs as I  # noqa: E402

pytestmark = pytest.mark.gpu
RES_TOL = 1e-8
SOL_TOL = 1e-6


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_01800_gb300 import api as A
    return A


def _noalloc(api, w, x, prec):
    L = api._lib.load()
    dx = np.ascontiguousarray(w.dx, dtype=np.float64)
    dy = np.ascontiguousarray(w.dy, dtype=np.float64)
    rhs = torch.tensor(w.f, dtype=torch.float64, device="cuda")
    info = api._lib.ppe_solve_info()
    st = L.ppe_solve_noalloc(w.nx, w.ny, dx.ctypes.data_as(ctypes.c_void_p), dy.ctypes.data_as(ctypes.c_void_p),
                             ctypes.c_void_p(rhs.data_ptr()), ctypes.c_void_p(x.data_ptr()), RES_TOL, prec,
                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), ctypes.byref(info))
    return st, info


def _ragged(nx, ny, seed):
    g = I.rng(seed)
    dx, dy = I.random_spacing(nx, g), I.random_spacing(ny, g)
    return I.Workload(f"ragged{nx}x{ny}", dx, dy, I.gaussian_rhs(dx, dy, g, 6))


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_noalloc_matches_regular_solve_twice(api, prec):
    p = api.PPE_PREC_MIXED if prec == "mixed" else api.PPE_PREC_FP64
    for w in (I.config1(4), _ragged(150, 97, 21)):       # two calls in a row, different systems
        grid = api.ppe_create_grid(w.dx, w.dy)
        x_ref = torch.zeros(w.ny, w.nx, dtype=torch.float64, device="cuda")
        api.ppe_solve(grid, torch.tensor(w.f, dtype=torch.float64, device="cuda"), x_ref, RES_TOL,
                      api.PPE_MODE_PCG, p)
        x = torch.full((w.ny, w.nx), 3.0, dtype=torch.float64, device="cuda")   # non-zero initial guess
        st, info = _noalloc(api, w, x, p)
        assert st == 0, api._lib.load().ppe_last_error()
        assert info.status == 0 and info.rel_res_true <= RES_TOL
        a, b = x.cpu().numpy(), x_ref.cpu().numpy()
        assert np.linalg.norm(a - b) / np.linalg.norm(b) <= SOL_TOL


@pytest.mark.parametrize("prec,shapes", [("mixed", ((256, 256), (512, 128))),
                                         ("fp64", ((256, 256), (4096, 16), (17, 3855)))])
def test_noalloc_at_the_size_limits(api, prec, shapes):
    """Grids that fill the fixed array, two or three calls in a row: 65,536
    cells as 256 x 256; a 4096 x 16 strip whose rows reach the width limit;
    and 17 x 3855, whose rows pad from 17 to 20 cells, so that the padded
    vectors come closest to their bound.  The long strips need tens of
    thousands of Jacobi-PCG iterations even in FP64 (the oracle takes 27,212
    on the 4096 x 16 one): there FP32 inner iterations stall whatever the
    entry point (ppe_solve then continues in FP64; this entry point reports
    PPE_ERR_NOT_CONVERGED), so mixed precision runs the 256 x 256 grid and a
    512 x 128 one."""
    p = api.PPE_PREC_MIXED if prec == "mixed" else api.PPE_PREC_FP64
    for k, (nx, ny) in enumerate(shapes):
        w = _ragged(nx, ny, 41 + 2 * k)
        grid = api.ppe_create_grid(w.dx, w.dy)
        x_ref = torch.zeros(w.ny, w.nx, dtype=torch.float64, device="cuda")
        api.ppe_solve(grid, torch.tensor(w.f, dtype=torch.float64, device="cuda"), x_ref, RES_TOL,
                      api.PPE_MODE_PCG, p)
        x = torch.zeros((w.ny, w.nx), dtype=torch.float64, device="cuda")
        st, info = _noalloc(api, w, x, p)
        assert st == 0, api._lib.load().ppe_last_error()
        assert info.status == 0 and info.rel_res_true <= RES_TOL
        a, b = x.cpu().numpy(), x_ref.cpu().numpy()
        assert np.linalg.norm(a - b) / np.linalg.norm(b) <= SOL_TOL


def test_noalloc_rejects_oversized_grid(api):
    n = 300                                             # 90000 cells > 65536
    w = I.Workload("big", I.uniform_spacing(n), I.uniform_spacing(n), np.zeros((n, n)))
    x = torch.zeros(n, n, dtype=torch.float64, device="cuda")
    st, _ = _noalloc(api, w, x, api.PPE_PREC_MIXED)
    assert st == api._lib.PPE_ERR_ARG
    assert b"65536" in api._lib.load().ppe_last_error()
