"""The two solve drivers and the per-phase report.

By default a solve -- one system or a batch, plain PCG or hybrid -- runs as
one CUDA graph launch whose device-side loop alternates solver segments and
network branches (ppe_solve_info.drive == 0).  opts.host_loop = 1 has the host
launch each segment instead (drive == 1).  Both drivers run the same kernels
on the same data in the same order, so their answers must agree bit for bit
(solution and iteration counts).  The hybrid batch is also checked against
the FP64 oracle, and the report's phase times must add up to at most the
call's time.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2604_01800_gb300 import inputs as I  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-8
WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2604_01800_gb300",
                       "weights", "hydea_mconv.ppenet")


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
    return I.Workload(f"ragged{nx}x{ny}", dx, dy, I.gaussian_rhs(dx, dy, g, 6))


def _solve(api, grid, w, mode, prec, host_loop, net=None, **opts):
    api.ppe_set_options(grid, host_loop=host_loop, **opts)     # the defaults plus these
    x = torch.zeros(w.ny, w.nx, dtype=torch.float64, device="cuda")
    info = api.ppe_solve(grid, _dev(w.f), x, TOL, mode, prec, net=net)
    return x.cpu().numpy(), info


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
@pytest.mark.parametrize("shape", [(64, 64), (150, 97), (512, 33)])
def test_graph_and_host_loop_agree_pcg(api, prec, shape):
    w = _ragged(*shape, 31 + shape[0])
    p = api.PPE_PREC_MIXED if prec == "mixed" else api.PPE_PREC_FP64
    grid = api.ppe_create_grid(w.dx, w.dy)
    xg, ig = _solve(api, grid, w, api.PPE_MODE_PCG, p, 0)
    xh, ih = _solve(api, grid, w, api.PPE_MODE_PCG, p, 1)
    assert ig["drive"] == 0 and ih["drive"] == 1
    assert ig["status"] == 0 and ig["iters_pcg"] == ih["iters_pcg"] and ig["refinements"] == ih["refinements"]
    assert np.array_equal(xg, xh)
    assert oracle.true_relres(w.dx, w.dy, w.f, xg) <= TOL * 1.05
    # a second graph solve reuses the graph and gives the same answer
    xg2, _ = _solve(api, grid, w, api.PPE_MODE_PCG, p, 0)
    assert np.array_equal(xg, xg2)


def test_graph_and_host_loop_agree_hybrid(api):
    """Hybrid solves with the shipped network: the device-side loop opens the
    network branch exactly when the host loop would run the network."""
    w = I.config3(1)
    net = api.net_load(WEIGHTS)
    grid = api.ppe_create_grid(w.dx, w.dy, w.mask)
    net.attach(grid)
    opts = dict(dlsm_stall_limit=0, hybrid_budget=40)
    xg, ig = _solve(api, grid, w, api.PPE_MODE_HYBRID, api.PPE_PREC_MIXED, 0, net, **opts)
    xh, ih = _solve(api, grid, w, api.PPE_MODE_HYBRID, api.PPE_PREC_MIXED, 1, net, **opts)
    assert ig["drive"] == 0 and ih["drive"] == 1
    assert ig["net_calls"] >= 8 and ig["net_calls"] == ih["net_calls"]
    assert (ig["iters_pcg"], ig["iters_dlsm"]) == (ih["iters_pcg"], ih["iters_dlsm"])
    assert np.array_equal(xg, xh)
    assert oracle.true_relres(w.dx, w.dy, w.f, xg) <= TOL * 1.05


def test_phase_times_add_up(api):
    w = I.config3(0)
    net = api.net_load(WEIGHTS)
    grid = api.ppe_create_grid(w.dx, w.dy, w.mask)
    net.attach(grid)
    api.ppe_set_options(grid, dlsm_stall_limit=0, hybrid_budget=30)
    x = torch.zeros(w.ny, w.nx, dtype=torch.float64, device="cuda")
    info = api.ppe_solve(grid, _dev(w.f), x, TOL, api.PPE_MODE_HYBRID, api.PPE_PREC_MIXED, net=net)
    parts = info["ms_pcg"] + info["ms_dlsm"] + info["ms_refine"] + info["ms_net"]
    assert min(info["ms_pcg"], info["ms_dlsm"], info["ms_refine"], info["ms_net"]) > 0, info
    assert parts <= info["ms_total"] * 1.02 and parts >= 0.5 * info["ms_total"], info


@pytest.mark.parametrize("mode", ["pcg", "hybrid"])
def test_batch_graph_and_host_loop_agree(api, mode):
    """Eight uneven systems in one batch: segments end on the step budget and
    the plan is re-drawn on the device (graph) or on the host (host loop) by the
    same planner, so both give identical answers."""
    ws = I.config4(8, nmin=64, nmax=200)
    grids = [api.ppe_create_grid(w.dx, w.dy, w.mask) for w in ws]
    m = api.PPE_MODE_HYBRID if mode == "hybrid" else api.PPE_MODE_PCG
    net = None
    if mode == "hybrid":
        net = api.net_load(WEIGHTS)
        for g in grids:
            net.attach(g)
    out = []
    for host_loop in (0, 1):
        for g in grids:
            api.ppe_set_options(g, host_loop=host_loop)
        rhs = [_dev(w.f) for w in ws]
        xs = [torch.zeros_like(r) for r in rhs]
        infos, st = api.ppe_solve_batch(grids, rhs, xs, TOL, m, api.PPE_PREC_MIXED, net=net)
        assert st == 0
        out.append(([x.cpu().numpy() for x in xs], infos))
    (xa, ia), (xb, ib) = out
    for k, w in enumerate(ws):
        assert ia[k]["drive"] == 0 and ib[k]["drive"] == 1
        assert (ia[k]["iters_pcg"], ia[k]["iters_dlsm"]) == (ib[k]["iters_pcg"], ib[k]["iters_dlsm"]), w.name
        assert np.array_equal(xa[k], xb[k]), w.name
        assert oracle.true_relres(w.dx, w.dy, w.f, xa[k]) <= TOL * 1.05
    if mode == "hybrid":
        assert sum(i["net_calls"] for i in ia) >= len(ws)


def test_replaced_network_is_not_replayed_from_a_stale_graph(api):
    """A grid's solve graph holds the attached network's forward pass.  After
    that network is destroyed, a new one attached to the same grid (whose
    object and buffers may reuse the freed memory) must get graphs of its
    own: its hybrid solve on the reused grid equals, bit for bit, the same
    solve on a fresh grid."""
    w = _ragged(64, 48, 21)
    cfg = api.net_default_config(widths=[16, 32], c_last=8, trunk_hidden=[16, 24], phi_hidden=4)
    opts = dict(dlsm_stall_limit=0, hybrid_budget=60)
    grid = api.ppe_create_grid(w.dx, w.dy)
    first = api.net_create(cfg, 11)
    first.attach(grid)
    _solve(api, grid, w, api.PPE_MODE_HYBRID, api.PPE_PREC_MIXED, 0, net=first, **opts)
    first.close()
    second = api.net_create(cfg, 12)
    second.attach(grid)
    xa, ia = _solve(api, grid, w, api.PPE_MODE_HYBRID, api.PPE_PREC_MIXED, 0, net=second, **opts)
    second.close()
    fresh = api.ppe_create_grid(w.dx, w.dy)
    again = api.net_create(cfg, 12)
    again.attach(fresh)
    xb, ib = _solve(api, fresh, w, api.PPE_MODE_HYBRID, api.PPE_PREC_MIXED, 0, net=again, **opts)
    assert ia["status"] == 0 and ib["status"] == 0 and ia["iters_dlsm"] >= 1
    assert (ia["iters_pcg"], ia["iters_dlsm"]) == (ib["iters_pcg"], ib["iters_dlsm"])
    assert np.array_equal(xa, xb)
    again.close()
    fresh.close()
    grid.close()
