"""The autotuner times the iteration-pass variants (the tile-cooperative pass
at each tile height, the streaming pass) on a grid and the solves that
follow use its choice; results stay within the parity bars."""
import json
import os

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


def test_autotune_then_solve(api, tmp_path):
    cache = tmp_path / "tune.jsonl"
    os.environ["PPE_TUNE_CACHE"] = str(cache)
    try:
        g = I.rng(31)
        dx, dy = I.random_spacing(700, g), I.random_spacing(500, g)
        f = I.gaussian_rhs(dx, dy, g, 6)
        grid = api.ppe_create_grid(dx, dy)
        rep = api.ppe_autotune(grid)
        assert rep["iter_pass"] in (1, 2) and rep["tile_rows"] in (4, 8, 16)
        assert all(v > 0 for v in rep["us_per_iter"].values()), rep
        best = min(rep["us_per_iter"].values())
        chosen = {1: "tile", 2: "stream"}[rep["iter_pass"]]
        assert rep["us_per_iter"][chosen] == best
        line = json.loads(cache.read_text().strip().splitlines()[-1])
        assert (line["nx"], line["ny"], line["iter_pass"], line["tile_rows"]) == (700, 500, rep["iter_pass"],
                                                                                rep["tile_rows"])
        # a solve with the default options now runs the tuned variant
        x = torch.zeros(500, 700, dtype=torch.float64, device="cuda")
        info = api.ppe_solve(grid, torch.tensor(f, device="cuda"), x, 1e-8, api.PPE_MODE_PCG, api.PPE_PREC_MIXED)
        assert info["status"] == 0
        assert oracle.true_relres(dx, dy, f, x.cpu().numpy()) <= 1.05e-8
    finally:
        os.environ.pop("PPE_TUNE_CACHE", None)


def test_autotune_small_grid_picks_a_tile_height(api, tmp_path):
    """On the 256^2 cylinder grid the tile-cooperative pass wins and the tuned
    height is one of the three; the tuned solve meets the parity bars."""
    os.environ["PPE_TUNE_CACHE"] = str(tmp_path / "tune.jsonl")
    try:
        w = I.config3(0)
        grid = api.ppe_create_grid(w.dx, w.dy)
        rep = api.ppe_autotune(grid)
        assert rep["iter_pass"] == 1 and rep["tile_rows"] in (4, 8, 16), rep
        x = torch.zeros(w.ny, w.nx, dtype=torch.float64, device="cuda")
        info = api.ppe_solve(grid, torch.tensor(w.f, device="cuda"), x, 1e-8, api.PPE_MODE_PCG, api.PPE_PREC_MIXED)
        assert info["status"] == 0
        assert oracle.true_relres(w.dx, w.dy, w.f, x.cpu().numpy()) <= 1.05e-8
    finally:
        os.environ.pop("PPE_TUNE_CACHE", None)


def test_batch_takes_a_shared_tuned_choice(api, tmp_path):
    """Two systems of one tuned shape (64^2): the batch runs the tuned pass and
    tile height for both, and each meets the parity bars."""
    os.environ["PPE_TUNE_CACHE"] = str(tmp_path / "tune.jsonl")
    try:
        ws = [I.config1(0), I.config1(1)]
        grids = [api.ppe_create_grid(w.dx, w.dy) for w in ws]
        rep = api.ppe_autotune(grids[0])            # the second grid finds the shape in the table
        assert rep["tile_rows"] in (4, 8, 16)
        rhs = [torch.tensor(w.f, device="cuda") for w in ws]
        xs = [torch.zeros(w.ny, w.nx, dtype=torch.float64, device="cuda") for w in ws]
        infos, st = api.ppe_solve_batch(grids, rhs, xs, 1e-8, api.PPE_MODE_PCG, api.PPE_PREC_MIXED)
        assert st == 0
        for w, x, info in zip(ws, xs, infos):
            assert info["status"] == 0
            assert oracle.true_relres(w.dx, w.dy, w.f, x.cpu().numpy()) <= 1.05e-8
    finally:
        os.environ.pop("PPE_TUNE_CACHE", None)
