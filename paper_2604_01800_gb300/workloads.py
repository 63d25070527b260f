"""Small, self-contained workloads for profiling one kernel at a time.

    python -m paper_2604_01800_gb300.workloads c2            # 512x512 refined box, mixed PCG to 1e-8
    python -m paper_2604_01800_gb300.workloads capped N ITS  # N x N box grid, mixed PCG capped at ITS iterations
    python -m paper_2604_01800_gb300.workloads infer         # network inference on the 256x256 cylinder grid
    python -m paper_2604_01800_gb300.workloads train N STEPS # training steps, batch 8 on an N x N stretched grid
    python -m paper_2604_01800_gb300.workloads hybrid        # hybrid solve (shipped network) on the 256x256 cylinder grid
    python -m paper_2604_01800_gb300.workloads mg NAME       # multigrid-partner solve: c1, c2, c3 or c5
    python -m paper_2604_01800_gb300.workloads pcg NAME      # plain mixed Jacobi PCG: c1, c2, c3 or c5

A trailing ``host`` (``hybrid host``, ``pcg c3 host``) runs the solves with
the host-loop driver, which launches the same solver kernel directly instead
of from the solve's CUDA graph (a profiler replays direct launches).

Each runs its solve (or inference) twice or more: the first launch warms up,
so a profiler can skip it (``-s 1``).  Synthetic inputs only.
"""
from __future__ import annotations

import sys

import numpy as np


def c2():
    import torch
    from . import api, inputs as I
    w = I.config2(0)
    g = api.ppe_create_grid(w.dx, w.dy)
    rhs = torch.tensor(w.f, dtype=torch.float64, device="cuda")
    for _ in range(2):
        x = torch.zeros_like(rhs)
        info = api.ppe_solve(g, rhs, x, 1e-8, api.PPE_MODE_PCG, api.PPE_PREC_MIXED)
    torch.cuda.synchronize()
    print(f"c2: {info['iters_pcg']} iterations, {info['ms_total']:.2f} ms")


def capped(n: int, its: int):
    import torch
    from . import api, inputs as I
    dx = I.box_spacing(n, 0.4, 0.6, 1.01)
    xc = np.cumsum(dx) - 0.5 * dx
    gx = np.cos(np.pi * xc) + 0.3 * np.cos(3 * np.pi * xc)
    gx -= np.dot(dx, gx) / dx.sum()
    g = api.ppe_create_grid(dx, dx)
    rhs = torch.outer(torch.tensor(gx, device="cuda"), torch.tensor(gx, device="cuda")).contiguous()
    x = torch.zeros_like(rhs)
    api.ppe_set_options(g, max_iters=its, inner_rtol=1e-12)
    for _ in range(2):
        x.zero_()
        info = api.ppe_solve(g, rhs, x, 1e-14, api.PPE_MODE_PCG, api.PPE_PREC_MIXED, raise_on_error=False)
    torch.cuda.synchronize()
    print(f"capped {n}x{n}: {info['iters_pcg']} iterations, {info['ms_total']:.2f} ms")


def infer():
    import torch
    from . import api, inputs as I
    w = I.config3(0)
    g = api.ppe_create_grid(w.dx, w.dy, w.mask)
    net = api.net_create(api.net_default_config(), 1)
    net.attach(g)
    r = torch.randn(w.ny, w.nx, device="cuda", dtype=torch.float32)
    e = torch.empty_like(r)
    for _ in range(3):
        net.infer(g, r, e)
    torch.cuda.synchronize()
    print(f"infer 256x256: |e| = {float(e.abs().mean()):.3e}")


def train(n: int, steps: int):
    import time

    import torch
    from . import api, inputs as I
    net = api.net_create(api.net_default_config(), 1)
    g = I.rng(3)
    dx, dy = I.random_spacing(n, g), I.random_spacing(n, g)
    grid = api.ppe_create_grid(dx, dy)
    net.attach(grid)
    R = np.stack([I.training_rhs(dx, dy, g) for _ in range(8)]).astype(np.float32)
    R /= np.linalg.norm(R.reshape(8, -1), axis=1)[:, None, None]
    Rt = torch.tensor(R, device="cuda")
    hp = api.net_default_hparams(lr0=1e-3, total_steps=max(steps, 1))
    for i in range(steps):
        torch.cuda.synchronize()
        t = time.perf_counter()
        loss = net.train_step(grid, Rt, hp)
        torch.cuda.synchronize()
        print(f"train {n}x{n} step {i}: loss {loss:.4e}, {1e3 * (time.perf_counter() - t):.1f} ms")


def hybrid(host: bool = False):
    import os

    import torch
    from . import api, inputs as I
    w = I.config3(0)
    g = api.ppe_create_grid(w.dx, w.dy, w.mask)
    net = api.net_load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "hydea_mconv.ppenet"))
    net.attach(g)
    api.ppe_set_options(g, host_loop=int(host))
    rhs = torch.tensor(w.f, dtype=torch.float64, device="cuda")
    for _ in range(2):
        x = torch.zeros_like(rhs)
        info = api.ppe_solve(g, rhs, x, 1e-8, api.PPE_MODE_HYBRID, api.PPE_PREC_MIXED, net=net)
    torch.cuda.synchronize()
    print(f"hybrid c3: {info['iters_pcg']} + {info['iters_dlsm']} iterations, {info['ms_total']:.2f} ms")


def _system(name: str):
    from . import inputs as I
    if name == "c5":
        dx, dy, bodies = I.config5_grid()
        return dx, dy, I.config5_rhs(0, dx, dy, bodies)
    w = {"c1": I.config1, "c2": I.config2, "c3": I.config3}[name](0)
    return w.dx, w.dy, w.f


def mg(name: str):
    import torch
    from . import api
    dx, dy, f = _system(name)
    g = api.ppe_create_grid(dx, dy)
    api.ppe_set_options(g, preconditioner=1)
    rhs = torch.tensor(f, dtype=torch.float64, device="cuda")
    for _ in range(2):
        x = torch.zeros_like(rhs)
        info = api.ppe_solve(g, rhs, x, 1e-8, api.PPE_MODE_PCG, api.PPE_PREC_MIXED)
    torch.cuda.synchronize()
    print(f"multigrid {name}: {info['iters_pcg']} iterations, {info['ms_total']:.2f} ms")


def pcg(name: str, host: bool = False):
    import torch
    from . import api
    dx, dy, f = _system(name)
    g = api.ppe_create_grid(dx, dy)
    api.ppe_set_options(g, host_loop=int(host))
    rhs = torch.tensor(f, dtype=torch.float64, device="cuda")
    for _ in range(2):
        x = torch.zeros_like(rhs)
        info = api.ppe_solve(g, rhs, x, 1e-8, api.PPE_MODE_PCG, api.PPE_PREC_MIXED)
    torch.cuda.synchronize()
    print(f"pcg {name}: {info['iters_pcg']} iterations, {info['ms_total']:.2f} ms")


def main(argv=None):
    a = sys.argv[1:] if argv is None else argv
    if not a or a[0] == "c2":
        c2()
    elif a[0] == "capped":
        capped(int(a[1]), int(a[2]))
    elif a[0] == "infer":
        infer()
    elif a[0] == "train":
        train(int(a[1]), int(a[2]))
    elif a[0] == "hybrid":
        hybrid(a[-1] == "host")
    elif a[0] == "mg":
        mg(a[1] if len(a) > 1 else "c2")
    elif a[0] == "pcg":
        pcg(a[1] if len(a) > 1 and a[1] != "host" else "c3", a[-1] == "host")
    else:
        raise SystemExit(__doc__)


if __name__ == "__main__":
    main()
