"""FP64 numpy oracle of the grid-spacing-aware DeepONet.  TEST INFRASTRUCTURE ONLY.

Restates, step by step and without fusion, what Sec. 2.4 defines:

* Multi-level distance-vector maps (Sec. 2.4, text after Eq. 17): the
  level-0 nodal coordinates are the cell centres; each deeper level takes a
  2x2 average pool of the previous level's coordinates.  At every node the
  four distances to the left / right / upper / lower neighbour form the
  4-channel map Delta_K.  At a wall the missing distance takes the value of
  the distance to the one interior neighbour on the same axis
  (nearest-neighbour padding).  Distances are scaled by the level-0 mean
  spacing of their axis (n / L).
* Mesh-Conv (Eqs. 16-17): eta = exp(-Phi(Delta)^2) per node, with Phi a
  pointwise 4 -> hidden -> 1 network (tanh hidden layer); the input feature
  map is multiplied by eta and then convolved (3x3, zero padding 1).
* Branch: a U-Net with two Mesh-Convs per encoder level, 2x2 average pooling
  between levels, nearest 2x up-sampling followed by a Mesh-Conv on the way
  up, concatenation [up-sampled, skip] and two Mesh-Convs per decoder level,
  GELU (erf form) after every convolution, then a 1x1 convolution to c_last
  features.
* Trunk: MLP on the normalised cell-centre coordinates (x/Lx, y/Ly), tanh
  hidden layers, linear output of c_last features.
* DeepONet output: sum_c branch_c * trunk_c + bias at every node.
* Loss (Eq. 18): mean over the batch and the N grid cells of
  (R - A NN(R))^2, A the volume-scaled operator of the CPU solver oracle.
* One optimiser step: SAM (perturbation rho * g / ||g||) followed by Adam
  on the gradient at the perturbed point, cosine learning-rate decay.

Grids whose size is not a multiple of 2^(levels-1)*2 are padded by repeating
the last cell width; the input is zero in the pad and the output is cropped.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

from . import CSR


# ---------------------------------------------------------------------------
# geometry: coordinates, distance maps, weight networks
# ---------------------------------------------------------------------------

def cell_centres(d):
    f = np.concatenate([[0.0], np.cumsum(np.asarray(d, dtype=np.float64))])
    return 0.5 * (f[:-1] + f[1:])


def level_coords(xc, levels):
    """Average-pooled coordinates for each U-Net level (tensor grid, so the
    2x2 pool of the coordinate map is the mean of two adjacent centres)."""
    out = [np.asarray(xc, dtype=np.float64)]
    for _ in range(1, levels):
        c = out[-1]
        out.append(0.5 * (c[0::2] + c[1::2]))
    return out


def side_distances(c):
    """(distance to previous node, distance to next node) with
    nearest-neighbour padding at both ends."""
    d = np.abs(np.diff(c))
    prev = np.concatenate([[d[0]], d])
    nxt = np.concatenate([d, [d[-1]]])
    return prev, nxt


def distance_maps(dx, dy, levels, sx=None, sy=None):
    """List of Delta_K arrays [4, H_K, W_K]; channels: left, right, up, down.

    ``dx``/``dy`` are the (padded) level-0 cell widths; distances are scaled
    by ``sx``/``sy`` (default nx/Lx and ny/Ly of the widths given)."""
    dx, dy = np.asarray(dx, np.float64), np.asarray(dy, np.float64)
    sx = dx.size / dx.sum() if sx is None else sx
    sy = dy.size / dy.sum() if sy is None else sy
    xs = level_coords(cell_centres(dx), levels)
    ys = level_coords(cell_centres(dy), levels)
    maps = []
    for xk, yk in zip(xs, ys):
        left, right = side_distances(xk)
        down, up = side_distances(yk)
        H, W = yk.size, xk.size
        D = np.empty((4, H, W))
        D[0] = (left * sx)[None, :]
        D[1] = (right * sx)[None, :]
        D[2] = (up * sy)[:, None]
        D[3] = (down * sy)[:, None]
        maps.append(D)
    return maps


def phi_forward(P, name, D):
    """Phi of one Mesh-Conv on a distance map D [4, H, W]; returns (phi, hidden)."""
    W1 = P[f"{name}.phi1.w"].astype(np.float64)
    b1 = P[f"{name}.phi1.b"].astype(np.float64)
    w2 = P[f"{name}.phi2.w"].astype(np.float64)
    b2 = float(P[f"{name}.phi2.b"][0])
    z = np.einsum("kc,chw->khw", W1, D) + b1[:, None, None]
    h = np.tanh(z)
    phi = np.einsum("k,khw->hw", w2, h) + b2
    return phi, h


def eta_map(P, name, D, mesh_conv=True):
    if not mesh_conv:
        return np.ones(D.shape[1:])
    phi, _ = phi_forward(P, name, D)
    return np.exp(-phi * phi)


# ---------------------------------------------------------------------------
# elementary operations (forward / backward)
# ---------------------------------------------------------------------------

def gelu(x):
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    cdf = 0.5 * (1.0 + erf(x / math.sqrt(2.0)))
    pdf = np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)
    return cdf + x * pdf


def conv3x3(X, Wt, b):
    """Cross-correlation with zero padding 1. X [B,Ci,H,W], Wt [Co,Ci,3,3]."""
    B, Ci, H, W = X.shape
    Xp = np.zeros((B, Ci, H + 2, W + 2))
    Xp[:, :, 1:-1, 1:-1] = X
    Y = np.zeros((B, Wt.shape[0], H, W))
    for ky in range(3):
        for kx in range(3):
            Y += np.einsum("oc,bchw->bohw", Wt[:, :, ky, kx], Xp[:, :, ky:ky + H, kx:kx + W])
    return Y + b[None, :, None, None]


def conv3x3_backward(X, Wt, dY):
    """Gradients of conv3x3 with respect to X, Wt and b."""
    B, Ci, H, W = X.shape
    Xp = np.zeros((B, Ci, H + 2, W + 2))
    Xp[:, :, 1:-1, 1:-1] = X
    dXp = np.zeros_like(Xp)
    dW = np.zeros_like(Wt)
    for ky in range(3):
        for kx in range(3):
            dXp[:, :, ky:ky + H, kx:kx + W] += np.einsum("oc,bohw->bchw", Wt[:, :, ky, kx], dY)
            dW[:, :, ky, kx] = np.einsum("bohw,bchw->oc", dY, Xp[:, :, ky:ky + H, kx:kx + W])
    return dXp[:, :, 1:-1, 1:-1], dW, dY.sum(axis=(0, 2, 3))


def avgpool2(X):
    return 0.25 * (X[:, :, 0::2, 0::2] + X[:, :, 1::2, 0::2] + X[:, :, 0::2, 1::2] + X[:, :, 1::2, 1::2])


def avgpool2_backward(dY):
    B, C, H, W = dY.shape
    dX = np.zeros((B, C, 2 * H, 2 * W))
    for a in range(2):
        for c in range(2):
            dX[:, :, a::2, c::2] = 0.25 * dY
    return dX


def upsample2(X):
    return X.repeat(2, axis=2).repeat(2, axis=3)


def upsample2_backward(dY):
    return dY[:, :, 0::2, 0::2] + dY[:, :, 1::2, 0::2] + dY[:, :, 0::2, 1::2] + dY[:, :, 1::2, 1::2]


# ---------------------------------------------------------------------------
# the network
# ---------------------------------------------------------------------------

def layer_list(widths):
    """(name, cin, cout, level) for every 3x3 Mesh-Conv, in execution order."""
    L = len(widths)
    out, cin = [], 1
    for k in range(L):
        out.append((f"enc{k}a", cin, widths[k], k))
        out.append((f"enc{k}b", widths[k], widths[k], k))
        cin = widths[k]
    for k in range(L - 2, -1, -1):
        out.append((f"up{k}", widths[k + 1], widths[k], k))
        out.append((f"dec{k}a", 2 * widths[k], widths[k], k))
        out.append((f"dec{k}b", widths[k], widths[k], k))
    return out


class Geometry:
    """Per-grid quantities the network needs: padded widths, distance maps,
    normalised trunk coordinates."""

    def __init__(self, dx, dy, levels, multiple=None):
        dx, dy = np.asarray(dx, np.float64), np.asarray(dy, np.float64)
        self.nx, self.ny = dx.size, dy.size
        self.lx, self.ly = dx.sum(), dy.sum()
        m = multiple or 2 ** levels
        self.dx = _pad(dx, m)
        self.dy = _pad(dy, m)
        self.W, self.H = self.dx.size, self.dy.size
        self.levels = levels
        # distance scale: inverse mean spacing of the unpadded grid
        self.sx, self.sy = self.nx / self.lx, self.ny / self.ly
        self.maps = distance_maps(self.dx, self.dy, levels, self.sx, self.sy)
        self.xn = cell_centres(self.dx) / self.lx
        self.yn = cell_centres(self.dy) / self.ly


def _pad(d, m):
    n = d.size
    k = -(-n // m) * m
    return d.copy() if k == n else np.concatenate([d, np.full(k - n, d[-1])])


def trunk_forward(P, geo, depth):
    """Trunk MLP on (x/Lx, y/Ly) at every padded node -> [C, H, W] plus cache."""
    H, W = geo.H, geo.W
    X = np.stack([np.broadcast_to(geo.xn[None, :], (H, W)),
                  np.broadcast_to(geo.yn[:, None], (H, W))]).reshape(2, -1)
    acts = [X]
    pre = []
    for i in range(depth):
        Wt = P[f"trunk{i}.w"].astype(np.float64)
        bt = P[f"trunk{i}.b"].astype(np.float64)
        z = Wt @ acts[-1] + bt[:, None]
        pre.append(z)
        acts.append(np.tanh(z) if i < depth - 1 else z)
    return acts[-1].reshape(-1, H, W), (acts, pre)


def trunk_backward(P, cache, dT, depth):
    acts, pre = cache
    g = {}
    d = dT.reshape(dT.shape[0], -1)
    for i in range(depth - 1, -1, -1):
        if i < depth - 1:
            d = d * (1.0 - np.tanh(pre[i]) ** 2)
        g[f"trunk{i}.w"] = d @ acts[i].T
        g[f"trunk{i}.b"] = d.sum(axis=1)
        d = P[f"trunk{i}.w"].astype(np.float64).T @ d
    return g


def forward(P, geo, R, widths, mesh_conv=True, trunk_depth=3):
    """NN(R) for a batch R [B, ny, nx] on geometry ``geo``; returns
    (e [B, ny, nx], cache)."""
    B = R.shape[0]
    X = np.zeros((B, 1, geo.H, geo.W))
    X[:, 0, :geo.ny, :geo.nx] = R
    cache = {"layers": {}, "X0": X}
    L = len(widths)
    etas = {}
    for name, ci, co, k in layer_list(widths):
        etas[name] = eta_map(P, name, geo.maps[k], mesh_conv)
    cache["etas"] = etas

    def mconv(name, Xin):
        Wt = P[f"{name}.w"].astype(np.float64)
        b = P[f"{name}.b"].astype(np.float64)
        Xb = Xin * etas[name][None, None]
        Z = conv3x3(Xb, Wt, b)
        cache["layers"][name] = (Xin, Xb, Z)
        return gelu(Z)

    x = X
    skips = []
    for k in range(L):
        if k > 0:
            x = avgpool2(x)
        x = mconv(f"enc{k}a", x)
        x = mconv(f"enc{k}b", x)
        skips.append(x)
    for k in range(L - 2, -1, -1):
        x = upsample2(x)
        x = mconv(f"up{k}", x)
        x = np.concatenate([x, skips[k]], axis=1)
        x = mconv(f"dec{k}a", x)
        x = mconv(f"dec{k}b", x)
    hfeat = x                                                    # [B, C0, H, W]
    Wh = P["head.w"].astype(np.float64)
    bh = P["head.b"].astype(np.float64)
    branch = np.einsum("kc,bchw->bkhw", Wh, hfeat) + bh[None, :, None, None]
    trunk, tcache = trunk_forward(P, geo, trunk_depth)
    e_full = np.einsum("bkhw,khw->bhw", branch, trunk) + float(P["out.b"][0])
    cache.update(hfeat=hfeat, branch=branch, trunk=trunk, tcache=tcache)
    return e_full[:, :geo.ny, :geo.nx], cache


def backward(P, geo, cache, de, widths, mesh_conv=True, trunk_depth=3):
    """Gradients of sum(de * e) with respect to every parameter."""
    B = de.shape[0]
    g = {}
    de_full = np.zeros((B, geo.H, geo.W))
    de_full[:, :geo.ny, :geo.nx] = de
    g["out.b"] = np.array([de_full.sum()])
    branch, trunk, hfeat = cache["branch"], cache["trunk"], cache["hfeat"]
    dbranch = de_full[:, None] * trunk[None]
    dtrunk = np.einsum("bhw,bkhw->khw", de_full, branch)
    g.update(trunk_backward(P, cache["tcache"], dtrunk, trunk_depth))
    Wh = P["head.w"].astype(np.float64)
    g["head.w"] = np.einsum("bkhw,bchw->kc", dbranch, hfeat)
    g["head.b"] = dbranch.sum(axis=(0, 2, 3))
    dx_ = np.einsum("kc,bkhw->bchw", Wh, dbranch)

    etas = cache["etas"]
    L = len(widths)

    def mconv_back(name, dout, k):
        Xin, Xb, Z = cache["layers"][name]
        dZ = dout * gelu_grad(Z)
        dXb, dW, db = conv3x3_backward(Xb, P[f"{name}.w"].astype(np.float64), dZ)
        g[f"{name}.w"] = dW
        g[f"{name}.b"] = db
        dXin = dXb * etas[name][None, None]
        if mesh_conv:
            deta = np.einsum("bchw,bchw->hw", dXb, Xin)
            phi, h = phi_forward(P, name, geo.maps[k])
            dphi = deta * etas[name] * (-2.0 * phi)
            w2 = P[f"{name}.phi2.w"].astype(np.float64)
            g[f"{name}.phi2.w"] = np.einsum("hw,khw->k", dphi, h)
            g[f"{name}.phi2.b"] = np.array([dphi.sum()])
            dz = (w2[:, None, None] * dphi[None]) * (1.0 - h * h)
            g[f"{name}.phi1.w"] = np.einsum("khw,chw->kc", dz, geo.maps[k])
            g[f"{name}.phi1.b"] = dz.sum(axis=(1, 2))
        else:
            for s in (".phi1.w", ".phi1.b", ".phi2.w", ".phi2.b"):
                g[name + s] = np.zeros(P[name + s].shape)
        return dXin

    dskips = [None] * L
    x = dx_
    for k in range(0, L - 1):
        x = mconv_back(f"dec{k}b", x, k)
        x = mconv_back(f"dec{k}a", x, k)
        cu = widths[k]
        dskips[k] = x[:, cu:]
        x = mconv_back(f"up{k}", x[:, :cu], k)
        x = upsample2_backward(x)
    for k in range(L - 1, -1, -1):
        if dskips[k] is not None:
            x = x + dskips[k]
        x = mconv_back(f"enc{k}b", x, k)
        x = mconv_back(f"enc{k}a", x, k)
        if k > 0:
            x = avgpool2_backward(x)
    return g


# ---------------------------------------------------------------------------
# loss (Eq. 18) and one SAM + Adam step
# ---------------------------------------------------------------------------

def loss_and_grad_e(A: CSR, R, e):
    """L = mean over batch and cells of (R - A e)^2 and dL/de
    (= -(2/(B N)) A^T (R - A e), A symmetric)."""
    B = R.shape[0]
    N = A.n
    res = np.stack([R[b].reshape(-1) - A.matvec(e[b]) for b in range(B)])
    L = float((res ** 2).sum() / (B * N))
    de = np.stack([-(2.0 / (B * N)) * A.matvec(res[b]) for b in range(B)])
    return L, de.reshape(e.shape)


def loss_and_grads(P, geo, A, R, widths, mesh_conv=True, trunk_depth=3):
    e, cache = forward(P, geo, R, widths, mesh_conv, trunk_depth)
    L, de = loss_and_grad_e(A, R, e)
    return L, backward(P, geo, cache, de, widths, mesh_conv, trunk_depth)


def cosine_lr(lr0, step, total):
    """Cosine decay from lr0 to 0 over ``total`` steps (step counts from 0)."""
    return 0.5 * lr0 * (1.0 + math.cos(math.pi * min(step, total) / total))


def sam_adam_step(P, state, geo, A, R, widths, hp, mesh_conv=True, trunk_depth=3):
    """One training step.  ``state`` holds Adam moments m, v and the step
    count t; ``hp`` = dict(lr0, total, rho, beta1, beta2, eps).  Returns
    (loss at the unperturbed point, new parameters, new state)."""
    names = list(P.keys())
    L0, g1 = loss_and_grads(P, geo, A, R, widths, mesh_conv, trunk_depth)
    gnorm = math.sqrt(sum(float((g1[n] ** 2).sum()) for n in names))
    scale = hp["rho"] / (gnorm + 1e-12)
    Pp = {n: P[n].astype(np.float64) + scale * g1[n] for n in names}
    _, g2 = loss_and_grads(Pp, geo, A, R, widths, mesh_conv, trunk_depth)
    t = state["t"] + 1
    lr = cosine_lr(hp["lr0"], state["t"], hp["total"])
    b1, b2, eps = hp["beta1"], hp["beta2"], hp["eps"]
    newP, m, v = {}, {}, {}
    for n in names:
        m[n] = b1 * state["m"][n] + (1 - b1) * g2[n]
        v[n] = b2 * state["v"][n] + (1 - b2) * g2[n] ** 2
        mh = m[n] / (1 - b1 ** t)
        vh = v[n] / (1 - b2 ** t)
        newP[n] = P[n].astype(np.float64) - lr * mh / (np.sqrt(vh) + eps)
    return L0, newP, {"m": m, "v": v, "t": t}


def adam_init(P):
    return {"m": {n: np.zeros(P[n].shape) for n in P},
            "v": {n: np.zeros(P[n].shape) for n in P}, "t": 0}
