"""Train the grid-spacing-aware DeepONet on the GPU with the library's own
forward/backward kernels (Sec. 2.4).

The training set is fabricated by the method itself: random stretched grids
(tanh or refined-box families, plus the cylinder-refined box family) and
unit-norm right-hand sides b = -V S whose sources S are Gaussian sums or
1/|k|^2 Fourier fields.  A step draws one grid and `batch` of its samples,
so the batch shares the grid's geometry caches.  Every `eval_every` steps
the hybrid solver is run on a held-out cylinder-grid system and its
iteration count is logged next to plain PCG's.

    python -m paper_2604_01800_gb300.train --steps 4000 --out weights.ppenet
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import time

import numpy as np

from . import inputs as I


def _make_grid(seed: int, sizes):
    g = I.rng(seed)
    n = int(sizes[int(g.integers(0, len(sizes)))])
    if g.uniform() < 0.25:     # cylinder-refined box family (the evaluation grid's family)
        cx, cy = g.uniform(0.3, 0.6), g.uniform(0.35, 0.65)
        w = g.uniform(0.2, 0.4)
        gr = g.uniform(1.02, 1.08)
        dx = I.box_spacing(n, max(0.05, cx - w / 2), min(0.95, cx + w / 2), gr)
        dy = I.box_spacing(n, max(0.05, cy - w / 2), min(0.95, cy + w / 2), gr)
    else:
        dx = I.random_spacing(n, g)
        dy = I.random_spacing(n, g)
    return dx, dy


def _samples(args):
    seed, dx, dy, count = args
    g = I.rng(seed)
    V = np.outer(dy, dx)
    out = np.empty((count, dy.size, dx.size), np.float32)
    for k in range(count):
        b = -V * I.training_rhs(dx, dy, g)
        b -= b.mean()
        out[k] = b / np.linalg.norm(b)
    return out


def build_dataset(n_grids: int, per_grid: int, sizes, seed: int = 7000, workers: int = 0):
    grids = [_make_grid(seed + i, sizes) for i in range(n_grids)]
    jobs = [(seed + 100000 + i, dx, dy, per_grid) for i, (dx, dy) in enumerate(grids)]
    workers = workers or min(16, os.cpu_count() or 1)
    if workers > 1:
        with mp.get_context("spawn").Pool(workers) as pool:
            data = pool.map(_samples, jobs)
    else:
        data = [_samples(j) for j in jobs]
    return grids, data


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--steps", type=int, default=4000)
    p.add_argument("--batch", type=int, default=8)
    p.add_argument("--grids", type=int, default=64)
    p.add_argument("--per-grid", type=int, default=320)
    p.add_argument("--sizes", default="128,160,192,224,256")
    p.add_argument("--lr", type=float, default=1e-3)
    p.add_argument("--rho", type=float, default=2e-4)
    p.add_argument("--eval-every", type=int, default=500)
    p.add_argument("--seed", type=int, default=1)
    p.add_argument("--out", default="hydea_mconv.ppenet")
    p.add_argument("--log", default=None)
    p.add_argument("--mesh-conv", type=int, default=1)
    a = p.parse_args(argv)

    sizes = [int(s) for s in a.sizes.split(",")]
    t0 = time.time()
    grids, data = build_dataset(a.grids, a.per_grid, sizes)
    t_data = time.time() - t0

    import torch

    from . import api
    dev = torch.device("cuda")
    net = api.net_create(api.net_default_config(mesh_conv=a.mesh_conv), a.seed)
    handles, pools = [], []
    for (dx, dy), R in zip(grids, data):
        gh = api.ppe_create_grid(dx, dy)
        net.attach(gh)
        handles.append(gh)
        pools.append(torch.tensor(R, device=dev))
    # held-out evaluation: the cylinder grid with a masked-divergence source
    w = I.config3(0)
    eg = api.ppe_create_grid(w.dx, w.dy, w.mask)
    net.attach(eg)
    erhs = torch.tensor(w.f, dtype=torch.float64, device=dev)

    def evaluate():
        x = torch.zeros_like(erhs)
        hyb = api.ppe_solve(eg, erhs, x, 1e-8, api.PPE_MODE_HYBRID, api.PPE_PREC_MIXED, net=net)
        x.zero_()
        pcg = api.ppe_solve(eg, erhs, x, 1e-8, api.PPE_MODE_PCG, api.PPE_PREC_MIXED)
        return {"hybrid_iters": hyb["iters_pcg"] + hyb["iters_dlsm"], "hybrid_dlsm": hyb["iters_dlsm"],
                "hybrid_ms": hyb["ms_total"], "pcg_iters": pcg["iters_pcg"], "pcg_ms": pcg["ms_total"]}

    hp = api.net_default_hparams(lr0=a.lr, total_steps=a.steps, rho=a.rho)
    gen = np.random.default_rng(a.seed)
    log = []
    t1 = time.time()
    ema = None
    for step in range(a.steps):
        gi = int(gen.integers(0, len(handles)))
        idx = torch.tensor(gen.choice(pools[gi].shape[0], a.batch, replace=False), device=dev)
        R = pools[gi].index_select(0, idx).contiguous()
        loss = net.train_step(handles[gi], R, hp)
        # loss relative to that of the zero network (mean R^2 = 1/N for unit-norm R)
        rel = loss * R[0].numel()
        ema = rel if ema is None else 0.98 * ema + 0.02 * rel
        if (step + 1) % a.eval_every == 0 or step == a.steps - 1:
            rec = {"step": step + 1, "rel_loss_ema": ema, "seconds": time.time() - t1}
            rec.update(evaluate())
            log.append(rec)
            print(json.dumps(rec), flush=True)
    net.save(a.out, with_moments=False)
    summary = {"steps": a.steps, "batch": a.batch, "grids": a.grids, "per_grid": a.per_grid, "sizes": sizes,
               "data_seconds": t_data, "train_seconds": time.time() - t1, "log": log}
    if a.log:
        with open(a.log, "w") as f:
            json.dump(summary, f, indent=1)
    return summary


if __name__ == "__main__":
    main()
