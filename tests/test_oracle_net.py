"""Pins of the network oracle (FP64 numpy) against closed forms, library
routines (torch CPU conv2d / avg_pool2d / interpolate / autograd / Adam) and
finite differences.

The torch re-statement below is written independently with library
primitives; agreement to rounding pins the oracle's hand-written loops,
its backward pass and its optimiser step.
"""
import math

import numpy as np
import pytest
import torch
import torch.nn.functional as F

import oracle
from oracle import net_oracle as N
from paper_2604_01800_gb300 import inputs as I


CFG = I.NetConfig(widths=(4, 6, 8), c_last=5, trunk=(7, 9), phi_hidden=3)


def _params(seed=1, phi_scale=0.5):
    P = I.net_params(CFG, seed, phi_scale=phi_scale)
    g = I.rng(seed + 100)
    for k in P:                          # nonzero biases so every term is exercised
        if k.endswith(".b"):
            P[k] = (0.1 * g.standard_normal(P[k].shape)).astype(np.float32)
    return P


def _grid(nx=13, ny=10, seed=3):
    g = I.rng(seed)
    return I.random_spacing(nx, g), I.random_spacing(ny, g)


# ---------------------------------------------------------------------------
# closed forms
# ---------------------------------------------------------------------------

def test_distance_maps_uniform_grid():
    n = 32
    d = I.uniform_spacing(n)
    maps = N.distance_maps(d, d, 4)
    for k, D in enumerate(maps):
        assert D.shape == (4, n >> k, n >> k)
        assert np.allclose(D, 2.0 ** k, rtol=0, atol=1e-12)


def test_distance_maps_nearest_padding_and_pooling():
    dx = np.array([0.1, 0.2, 0.3, 0.4])
    dy = np.array([1.0, 1.0, 2.0, 4.0])
    maps = N.distance_maps(dx, dy, 2, sx=1.0, sy=1.0)
    xc = np.array([0.05, 0.2, 0.45, 0.8])
    D0 = maps[0]
    assert np.allclose(D0[0, 0], [0.15, 0.15, 0.25, 0.35])        # left
    assert np.allclose(D0[1, 0], [0.15, 0.25, 0.35, 0.35])        # right
    assert np.allclose(D0[3, :, 0], [1.0, 1.0, 1.5, 3.0])         # down
    assert np.allclose(D0[2, :, 0], [1.0, 1.5, 3.0, 3.0])         # up
    x1 = [(xc[0] + xc[1]) / 2, (xc[2] + xc[3]) / 2]
    assert np.allclose(maps[1][0, 0], [x1[1] - x1[0]] * 2)


def test_eta_is_one_for_zero_phi():
    P = _params()
    for k in P:
        if ".phi2" in k:
            P[k][...] = 0
    D = N.distance_maps(*_grid(16, 16), 3)[0]
    assert np.all(N.eta_map(P, "enc0a", D) == 1.0)


# ---------------------------------------------------------------------------
# torch re-statement (library primitives)
# ---------------------------------------------------------------------------

def _torch_forward(P, dx, dy, R, mesh_conv=True):
    geo = N.Geometry(dx, dy, CFG.levels)
    T = {k: torch.tensor(v.astype(np.float64), dtype=torch.float64, requires_grad=True) for k, v in P.items()}
    H, W = geo.H, geo.W
    x = torch.zeros(R.shape[0], 1, H, W, dtype=torch.float64)
    x[:, 0, :geo.ny, :geo.nx] = torch.tensor(R, dtype=torch.float64)
    maps = [torch.tensor(m, dtype=torch.float64) for m in geo.maps]

    def eta(name, k):
        if not mesh_conv:
            return torch.ones(maps[k].shape[1:], dtype=torch.float64)
        D = maps[k].permute(1, 2, 0)                       # [H, W, 4]
        h = torch.tanh(F.linear(D, T[f"{name}.phi1.w"], T[f"{name}.phi1.b"]))
        phi = (h * T[f"{name}.phi2.w"]).sum(-1) + T[f"{name}.phi2.b"]
        return torch.exp(-phi ** 2)

    def mconv(name, k, inp):
        y = F.conv2d(inp * eta(name, k), T[f"{name}.w"], T[f"{name}.b"], padding=1)
        return F.gelu(y)

    skips = []
    for k in range(CFG.levels):
        if k:
            x = F.avg_pool2d(x, 2)
        x = mconv(f"enc{k}b", k, mconv(f"enc{k}a", k, x))
        skips.append(x)
    for k in range(CFG.levels - 2, -1, -1):
        x = mconv(f"up{k}", k, F.interpolate(x, scale_factor=2, mode="nearest"))
        x = torch.cat([x, skips[k]], 1)
        x = mconv(f"dec{k}b", k, mconv(f"dec{k}a", k, x))
    branch = F.conv2d(x, T["head.w"][:, :, None, None], T["head.b"])
    xy = torch.stack(torch.meshgrid(torch.tensor(geo.yn, dtype=torch.float64), torch.tensor(geo.xn, dtype=torch.float64),
                                   indexing="ij")[::-1], -1)
    t = xy
    depth = len(CFG.trunk) + 1
    for i in range(depth):
        t = F.linear(t, T[f"trunk{i}.w"], T[f"trunk{i}.b"])
        if i < depth - 1:
            t = torch.tanh(t)
    e = (branch * t.permute(2, 0, 1)[None]).sum(1) + T["out.b"]
    return e[:, :geo.ny, :geo.nx], T


@pytest.mark.parametrize("mesh_conv", [True, False])
def test_forward_matches_torch(mesh_conv):
    dx, dy = _grid()
    P = _params()
    R = I.rng(5).standard_normal((2, dy.size, dx.size))
    geo = N.Geometry(dx, dy, CFG.levels)
    e, _ = N.forward(P, geo, R, CFG.widths, mesh_conv, len(CFG.trunk) + 1)
    et, _ = _torch_forward(P, dx, dy, R, mesh_conv)
    assert np.allclose(e, et.detach().numpy(), rtol=1e-12, atol=1e-12 * np.abs(e).max())


def test_conv_without_eta_is_library_conv():
    g = I.rng(9)
    X = g.standard_normal((2, 3, 8, 5))
    Wt = g.standard_normal((4, 3, 3, 3))
    b = g.standard_normal(4)
    Y = N.conv3x3(X, Wt, b)
    Yt = F.conv2d(torch.tensor(X, dtype=torch.float64), torch.tensor(Wt, dtype=torch.float64),
                  torch.tensor(b, dtype=torch.float64), padding=1).numpy()
    assert np.allclose(Y, Yt, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("mesh_conv", [True, False])
def test_backward_matches_autograd(mesh_conv):
    dx, dy = _grid()
    P = _params(2)
    geo = N.Geometry(dx, dy, CFG.levels)
    A = oracle.CSR(dx, dy)
    R = I.rng(6).standard_normal((2, dy.size, dx.size))
    L, g = N.loss_and_grads(P, geo, A, R, CFG.widths, mesh_conv, len(CFG.trunk) + 1)
    et, T = _torch_forward(P, dx, dy, R, mesh_conv)
    Ad = torch.tensor(A.dense(), dtype=torch.float64)
    res = torch.tensor(R, dtype=torch.float64).reshape(2, -1) - et.reshape(2, -1) @ Ad.T
    Lt = (res ** 2).mean()
    Lt.backward()
    assert abs(L - Lt.item()) <= 1e-12 * abs(L)
    gmax = max(float(np.abs(v.grad.numpy()).max()) for v in T.values() if v.grad is not None)
    for k, v in T.items():
        ref = v.grad.numpy() if v.grad is not None else np.zeros(v.shape)
        # out.b has an exactly-zero gradient (A 1 = 0): compare on the global scale
        assert np.allclose(g[k], ref, rtol=1e-9, atol=1e-12 * gmax), k


def test_backward_finite_differences():
    dx, dy = _grid(16, 8, seed=4)
    P = {k: v.astype(np.float64) for k, v in _params(3).items()}
    geo = N.Geometry(dx, dy, CFG.levels)
    A = oracle.CSR(dx, dy)
    R = I.rng(8).standard_normal((1, dy.size, dx.size))
    depth = len(CFG.trunk) + 1
    _, g = N.loss_and_grads(P, geo, A, R, CFG.widths, True, depth)
    for name in ["enc0a.w", "dec0b.w", "up1.b", "enc2b.phi1.w", "dec1a.phi2.b", "head.w", "trunk1.w", "trunk2.b"]:
        # the largest-magnitude entry, so the difference quotient resolves it
        idx = np.unravel_index(int(np.argmax(np.abs(g[name]))), P[name].shape)
        h = 1e-5 * max(1.0, abs(P[name][idx]))
        Pp = {k: v.copy() for k, v in P.items()}
        Pm = {k: v.copy() for k, v in P.items()}
        Pp[name][idx] += h
        Pm[name][idx] -= h
        Lp = N.loss_and_grads(Pp, geo, A, R, CFG.widths, True, depth)[0]
        Lm = N.loss_and_grads(Pm, geo, A, R, CFG.widths, True, depth)[0]
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - g[name][idx]) <= 1e-6 * abs(fd), name


def test_loss_vanishes_at_exact_error():
    """Eq. 18: if NN(R) solves A e = R exactly, the loss is zero."""
    dx, dy = _grid(12, 12, seed=5)
    S = I.rng(2).standard_normal((12, 12))
    V = np.outer(dy, dx)
    S -= (V * S).sum() / V.sum()
    A = oracle.CSR(dx, dy)
    R = oracle.scaled_rhs(dx, dy, S)
    R -= R.mean()
    e, _, st = oracle.solve(dx, dy, S, tol_rel=1e-13)
    L, de = N.loss_and_grad_e(A, R[None], e[None])
    assert L <= 1e-24 * (R ** 2).mean()


def test_sam_adam_step_matches_torch_optimizer():
    dx, dy = _grid(16, 16, seed=6)
    P = _params(4)
    geo = N.Geometry(dx, dy, CFG.levels)
    A = oracle.CSR(dx, dy)
    R = I.rng(11).standard_normal((2, 16, 16))
    hp = dict(lr0=2e-3, total=10, rho=0.05, beta1=0.9, beta2=0.999, eps=1e-8)
    depth = len(CFG.trunk) + 1
    state = N.adam_init(P)
    Pcur = {k: v.astype(np.float64) for k, v in P.items()}
    # two steps to exercise bias correction and the cosine schedule
    for _ in range(2):
        L0, Pcur, state = N.sam_adam_step(Pcur, state, geo, A, R, CFG.widths, hp, True, depth)

    # torch: SAM by hand around torch.optim.Adam with a cosine schedule
    Ad = torch.tensor(A.dense(), dtype=torch.float64)
    T = {k: torch.tensor(v.astype(np.float64), dtype=torch.float64, requires_grad=True) for k, v in P.items()}
    opt = torch.optim.Adam(T.values(), lr=hp["lr0"], betas=(hp["beta1"], hp["beta2"]), eps=hp["eps"])
    sched = torch.optim.lr_scheduler.CosineAnnealingLR(opt, T_max=hp["total"], eta_min=0.0)

    def loss_of(Pd):
        et, TT = _torch_forward(Pd, dx, dy, R)
        res = torch.tensor(R, dtype=torch.float64).reshape(2, -1) - et.reshape(2, -1) @ Ad.T
        return (res ** 2).mean(), TT

    for _ in range(2):
        cur = {k: v.detach().numpy() for k, v in T.items()}
        L, TT = loss_of(cur)
        gr = torch.autograd.grad(L, list(TT.values()))
        gn = math.sqrt(sum(float((x ** 2).sum()) for x in gr))
        pert = {k: cur[k] + hp["rho"] / (gn + 1e-12) * gi.numpy() for k, gi in zip(TT, gr)}
        L2, TT2 = loss_of(pert)
        gr2 = torch.autograd.grad(L2, list(TT2.values()))
        opt.zero_grad()
        for (k, v), gi in zip(T.items(), gr2):
            v.grad = gi.clone()
        opt.step()
        sched.step()
    for k in P:
        ref = T[k].detach().numpy()
        assert np.allclose(Pcur[k], ref, rtol=1e-9, atol=1e-12), k
