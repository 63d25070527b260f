"""Train the grid-spacing-aware DeepONet on the GPU with the library's own
forward/backward kernels (Sec. 2.4).

The training set is fabricated by the method itself: random stretched grids
(tanh or refined-box families, plus the cylinder-refined box family) and
unit-norm right-hand sides b = -V S whose sources S are Gaussian sums or
1/|k|^2 Fourier fields.  A fraction of the samples is replaced by the
residual that plain PCG leaves on that system after k iterations (k
log-uniform), i.e. by the kind of residual a DLSM step receives in the
middle of a solve.  A step draws one grid and `batch` of its samples, so the
batch shares the grid's geometry caches.  Every `eval_every` steps
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


def pcg_residuals(api, grid, dx, dy, R, gen, frac, kmax, dev):
    """Replace a fraction of the unit-norm samples R (in place) by the
    normalised residual of k plain-PCG iterations on A x = R."""
    import torch
    V = np.outer(dy, dx)
    S = torch.empty(R.shape[1:], dtype=torch.float64, device=dev)
    x = torch.empty_like(S)
    r = torch.empty_like(S)
    for i in range(R.shape[0]):
        if gen.uniform() >= frac:
            continue
        k = int(np.exp(gen.uniform(0.0, np.log(kmax))))
        S.copy_(torch.from_numpy(-R[i].astype(np.float64) / V))
        x.zero_()
        api.ppe_set_options(grid, max_iters=max(1, k))
        api.ppe_solve(grid, S, x, 1e-14, api.PPE_MODE_PCG, api.PPE_PREC_MIXED, raise_on_error=False)
        api.ppe_residual(grid, S, x, r)
        rn = r.cpu().numpy()
        rn -= rn.mean()
        nrm = np.linalg.norm(rn)
        if nrm > 0:
            R[i] = (rn / nrm).astype(np.float32)
    api.ppe_set_options(grid)


def ritz_vectors(api, grid, n_cells: int, m: int, seed: int, dev):
    """Ritz vectors of the grid's operator A from m Lanczos steps with full
    reorthogonalisation (Sec. 2.3, Eq. 13: T_m = V_m^T A V_m, Q_m = V_m U_m),
    ordered by increasing Ritz value; the constant null space is projected
    out.  Returns (Q [m, N] FP32 on the device, Ritz values)."""
    import torch
    gen = torch.Generator(device=dev).manual_seed(seed)
    V = torch.zeros(m, n_cells, dtype=torch.float64, device=dev)
    v = torch.randn(n_cells, dtype=torch.float64, device=dev, generator=gen)
    v -= v.mean()
    v /= v.norm()
    w = torch.empty_like(v)
    alpha = np.zeros(m)
    beta = np.zeros(m)
    ny, nx = grid.ny, grid.nx
    k_used = m
    for k in range(m):
        V[k] = v
        api.ppe_apply(grid, v.view(ny, nx), w.view(ny, nx))
        alpha[k] = float(w @ v)
        w -= alpha[k] * v
        if k > 0:
            w -= beta[k - 1] * V[k - 1]
        for _ in range(2):                      # full reorthogonalisation, twice
            w -= V[:k + 1].t() @ (V[:k + 1] @ w)
        w -= w.mean()
        beta[k] = float(w.norm())
        if beta[k] < 1e-12 * abs(alpha[k]):
            k_used = k + 1
            break
        v = w / beta[k]
    T = np.diag(alpha[:k_used]) + np.diag(beta[:k_used - 1], 1) + np.diag(beta[:k_used - 1], -1)
    theta, U = np.linalg.eigh(T)
    Q = torch.tensor(U.T, device=dev) @ V[:k_used]
    return Q.float(), theta


def ritz_samples(Q, count: int, b: float, gen):
    """Samples of Eqs. 14-15: R = sum_j c_j q_j / ||.||, c_j = 9 N(0,1) for the
    lowest b*m Ritz vectors and N(0,1) for the others."""
    import torch
    m = Q.shape[0]
    c = torch.tensor(gen.standard_normal((count, m)), dtype=torch.float32, device=Q.device)
    c[:, :int(b * m)] *= 9.0
    R = c @ Q
    R -= R.mean(dim=1, keepdim=True)
    return R / R.norm(dim=1, keepdim=True)


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
    p.add_argument("--pcg-frac", type=float, default=0.7)
    p.add_argument("--pcg-kmax", type=int, default=2000)
    p.add_argument("--init", default=None, help="start from this weights file")
    p.add_argument("--ritz-c3", type=int, default=0,
                   help="fine-tune on the 256x256 cylinder grid with Ritz-vector samples (Eqs. 13-15) "
                        "from this many Lanczos steps instead of the random-grid dataset")
    p.add_argument("--ritz-b", type=float, default=0.6)
    a = p.parse_args(argv)

    sizes = [int(s) for s in a.sizes.split(",")]
    t0 = time.time()
    if a.ritz_c3:
        grids, data = [], []
    else:
        grids, data = build_dataset(a.grids, a.per_grid, sizes)
    t_data = time.time() - t0

    import torch

    from . import api
    dev = torch.device("cuda")
    net = api.net_load(a.init) if a.init else api.net_create(api.net_default_config(mesh_conv=a.mesh_conv), a.seed)
    handles, pools = [], []
    rgen = np.random.default_rng(a.seed + 17)
    t_pcg = time.time()
    for (dx, dy), R in zip(grids, data):
        gh = api.ppe_create_grid(dx, dy)
        if a.pcg_frac > 0:
            pcg_residuals(api, gh, dx, dy, R, rgen, a.pcg_frac, a.pcg_kmax, dev)
        net.attach(gh)
        handles.append(gh)
        pools.append(torch.tensor(R, device=dev))
    t_data += time.time() - t_pcg
    # held-out evaluation: the cylinder grid with a masked-divergence source
    w = I.config3(0)
    eg = api.ppe_create_grid(w.dx, w.dy, w.mask)
    net.attach(eg)
    erhs = torch.tensor(w.f, dtype=torch.float64, device=dev)
    ritz_Q = None
    if a.ritz_c3:
        t_r = time.time()
        ritz_Q, theta = ritz_vectors(api, eg, w.nx * w.ny, a.ritz_c3, a.seed + 5, dev)
        t_data += time.time() - t_r
        print(json.dumps({"ritz_steps": a.ritz_c3, "ritz_min": float(theta[0]), "ritz_max": float(theta[-1]),
                          "seconds": time.time() - t_r}), flush=True)

    def evaluate():
        out = {}
        for keep in (0, 1):
            api.ppe_set_options(eg, keep_dir_after_dlsm=keep)
            x = torch.zeros_like(erhs)
            hyb = api.ppe_solve(eg, erhs, x, 1e-8, api.PPE_MODE_HYBRID, api.PPE_PREC_MIXED, net=net,
                                raise_on_error=False)
            out[f"hybrid{keep}"] = [hyb["iters_pcg"] + hyb["iters_dlsm"], hyb["iters_dlsm"], round(hyb["ms_total"], 2),
                                    hyb["fell_back"], hyb["status"]]
        x = torch.zeros_like(erhs)
        pcg = api.ppe_solve(eg, erhs, x, 1e-8, api.PPE_MODE_PCG, api.PPE_PREC_MIXED)
        out["pcg"] = [pcg["iters_pcg"], round(pcg["ms_total"], 2)]
        return out

    hp = api.net_default_hparams(lr0=a.lr, total_steps=a.steps, rho=a.rho)
    gen = np.random.default_rng(a.seed)
    log = []
    t1 = time.time()
    ema = None
    for step in range(a.steps):
        if ritz_Q is not None:
            gh = eg
            R = ritz_samples(ritz_Q, a.batch, a.ritz_b, gen).view(a.batch, w.ny, w.nx).contiguous()
        else:
            gi = int(gen.integers(0, len(handles)))
            idx = torch.tensor(gen.choice(pools[gi].shape[0], a.batch, replace=False), device=dev)
            R = pools[gi].index_select(0, idx).contiguous()
            gh = handles[gi]
        loss = net.train_step(gh, R, hp)
        # loss relative to that of the zero network (mean R^2 = 1/N for unit-norm R)
        rel = loss * R[0].numel()
        ema = rel if ema is None else 0.98 * ema + 0.02 * rel
        if (step + 1) % a.eval_every == 0 or step == a.steps - 1:
            rec = {"step": step + 1, "rel_loss_ema": ema, "seconds": time.time() - t1}
            rec.update(evaluate())
            log.append(rec)
            print(json.dumps(rec), flush=True)
            net.save(a.out, with_moments=False)     # checkpoint
    net.save(a.out, with_moments=False)
    summary = {"steps": a.steps, "batch": a.batch, "grids": a.grids, "per_grid": a.per_grid, "sizes": sizes,
               "data_seconds": t_data, "train_seconds": time.time() - t1, "log": log}
    if a.log:
        with open(a.log, "w") as f:
            json.dump(summary, f, indent=1)
    return summary


if __name__ == "__main__":
    main()
