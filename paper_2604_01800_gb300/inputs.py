"""Seeded synthetic inputs for the pressure Poisson equation (PPE) hot path.

This module draws grids, right-hand sides, obstacle masks and network
parameters.  It holds none of the solver's or the network's arithmetic: it
only produces the arrays that both the CUDA path and the CPU oracle consume,
so both sides see bit-identical inputs.

Every random draw goes through ``numpy.random.Generator(Philox(seed))`` so a
workload is fixed by its integer seed alone.

Grids are tensor-product, cell-centred, non-uniform Cartesian grids described
by 1-D cell widths ``dx[nx]`` and ``dy[ny]`` (Sec. 2.1 and the grids of
Sec. 3: a uniformly refined box around the body with progressive coarsening
toward the walls).  Fields are row-major ``[ny][nx]`` with ``x`` contiguous.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "rng", "uniform_spacing", "tanh_spacing", "box_spacing", "centres",
    "spacing_ratio", "gaussian_rhs", "fourier_rhs", "Body", "body_mask",
    "mask_rhs", "random_spacing", "random_bodies", "Workload",
    "config1", "config2", "config3", "config4", "config5_grid",
    "config5_rhs", "training_rhs", "NetConfig", "net_param_shapes",
    "net_params", "pad_spacing",
]


def rng(seed: int) -> np.random.Generator:
    """Counter-based generator (Philox-4x64) keyed by ``seed``."""
    return np.random.Generator(np.random.Philox(key=int(seed)))


# ---------------------------------------------------------------------------
# 1-D spacings
# ---------------------------------------------------------------------------

def uniform_spacing(n: int, length: float = 1.0) -> np.ndarray:
    return np.full(n, length / n, dtype=np.float64)


def tanh_spacing(n: int, beta: float, length: float = 1.0) -> np.ndarray:
    """Cells clustered toward both walls.

    Faces sit at ``L/2 * (1 + tanh(beta*(2*xi-1))/tanh(beta))`` for
    ``xi = k/n``, ``k = 0..n``; the widths are the face differences.
    """
    xi = np.arange(n + 1, dtype=np.float64) / n
    faces = 0.5 * length * (1.0 + np.tanh(beta * (2.0 * xi - 1.0)) / math.tanh(beta))
    faces[0], faces[-1] = 0.0, length
    return np.diff(faces)


def _geometric_count(h: float, gap: float, growth: float) -> int:
    """Number of cells h*g, h*g^2, ... whose total is closest to ``gap``."""
    if gap <= 0.0:
        return 0
    m = math.log1p(gap * (growth - 1.0) / (h * growth)) / math.log(growth)
    return max(1, int(round(m)))


def box_spacing(n: int, a: float, b: float, growth: float,
                length: float = 1.0) -> np.ndarray:
    """Uniform cells on ``[a, b]``, geometric coarsening toward both walls.

    The refined box holds ``n_in`` cells of width ``h = (b-a)/n_in``.  Each
    side outside it holds ``m`` cells of widths ``h*g^k`` (``k = 1..m``),
    rescaled as a whole so that the outermost face lands on the wall.  ``n_in``
    is the largest count for which the total is ``n``; any shortfall goes to
    the wider side.
    """
    assert 0.0 <= a < b <= length and growth > 1.0 and n >= 4
    left_gap, right_gap = a, length - b

    def total(n_in: int):
        h = (b - a) / n_in
        ml = _geometric_count(h, left_gap, growth)
        mr = _geometric_count(h, right_gap, growth)
        return n_in + ml + mr, ml, mr

    best = None
    for n_in in range(n, 0, -1):
        t, ml, mr = total(n_in)
        if t <= n:
            best = (n_in, ml, mr, t)
            break
    assert best is not None
    n_in, ml, mr, t = best
    short = n - t
    while short > 0:                       # pad the wider gap first
        if (left_gap >= right_gap and left_gap > 0) or right_gap <= 0:
            ml += 1
        else:
            mr += 1
        short -= 1
    h = (b - a) / n_in

    def side(m: int, gap: float) -> np.ndarray:
        if m == 0:
            return np.zeros(0)
        w = h * growth ** np.arange(1, m + 1, dtype=np.float64)
        return w * (gap / w.sum())

    left = side(ml, left_gap)[::-1]
    right = side(mr, right_gap)
    dx = np.concatenate([left, np.full(n_in, h), right])
    assert dx.size == n
    return dx


def centres(d: np.ndarray, origin: float = 0.0) -> np.ndarray:
    """Cell-centre coordinates for widths ``d``."""
    faces = origin + np.concatenate([[0.0], np.cumsum(d)])
    return 0.5 * (faces[:-1] + faces[1:])


def spacing_ratio(dx: np.ndarray, dy: np.ndarray) -> float:
    both = np.concatenate([dx, dy])
    return float(both.max() / both.min())


def pad_spacing(d: np.ndarray, multiple: int) -> np.ndarray:
    """Extend ``d`` to a multiple of ``multiple`` cells by repeating the last
    width (the network's grid padding)."""
    n = d.size
    m = -(-n // multiple) * multiple
    if m == n:
        return d.copy()
    return np.concatenate([d, np.full(m - n, d[-1])])


# ---------------------------------------------------------------------------
# Right-hand sides (the source S of M dp = S)
# ---------------------------------------------------------------------------

def _zero_volume_mean(f: np.ndarray, dx: np.ndarray, dy: np.ndarray) -> np.ndarray:
    vol = np.outer(dy, dx)
    return f - (vol * f).sum() / vol.sum()


def gaussian_rhs(dx, dy, g: np.random.Generator, n_gauss: int = 8,
                 sigma=(0.02, 0.2), amp=(0.5, 1.0), lx=1.0, ly=1.0):
    """Sum of Gaussians with seeded centres, widths and signed amplitudes,
    made compatible (zero volume-weighted mean)."""
    xc, yc = centres(dx), centres(dy)
    f = np.zeros((dy.size, dx.size))
    for _ in range(n_gauss):
        cx, cy = g.uniform(0, lx), g.uniform(0, ly)
        s = g.uniform(*sigma)
        a = g.uniform(*amp) * (1.0 if g.uniform() < 0.5 else -1.0)
        gx = np.exp(-((xc - cx) ** 2) / (2 * s * s))
        gy = np.exp(-((yc - cy) ** 2) / (2 * s * s))
        f += a * np.outer(gy, gx)
    return _zero_volume_mean(f, dx, dy)


def fourier_rhs(dx, dy, g: np.random.Generator, kmax: int = 32,
                lx=1.0, ly=1.0):
    """Random Fourier field: modes ``1 <= |k| <= kmax`` with amplitude
    ``a_k/|k|^2`` (``a_k ~ N(0,1)``), phases ``U(0, 2pi)``; zero mean."""
    xc, yc = centres(dx) / lx, centres(dy) / ly
    ks = [(kx, ky) for kx in range(kmax + 1) for ky in range(kmax + 1)
          if 1 <= math.hypot(kx, ky) <= kmax]
    kx = np.array([k[0] for k in ks], dtype=np.float64)
    ky = np.array([k[1] for k in ks], dtype=np.float64)
    a = g.standard_normal(len(ks)) / (kx * kx + ky * ky)
    phi = g.uniform(0, 2 * np.pi, len(ks))
    psi = g.uniform(0, 2 * np.pi, len(ks))
    cx = np.cos(np.pi * kx[:, None] * xc[None, :] + phi[:, None])   # [K, nx]
    cy = np.cos(np.pi * ky[:, None] * yc[None, :] + psi[:, None])   # [K, ny]
    f = (cy * a[:, None]).T @ cx                                    # [ny, nx]
    return _zero_volume_mean(f, dx, dy)


# ---------------------------------------------------------------------------
# Immersed bodies: mask and the masked-divergence right-hand side
# ---------------------------------------------------------------------------

@dataclass
class Body:
    """Circle (``a == b``) or ellipse with semi-axes ``a``, ``b`` rotated by
    ``angle`` about its centre."""
    cx: float
    cy: float
    a: float
    b: float
    angle: float = 0.0

    def level(self, x, y):
        """Approximate signed distance (negative inside)."""
        c, s = math.cos(self.angle), math.sin(self.angle)
        xr = (x - self.cx) * c + (y - self.cy) * s
        yr = -(x - self.cx) * s + (y - self.cy) * c
        rho = np.sqrt((xr / self.a) ** 2 + (yr / self.b) ** 2)
        return (rho - 1.0) * min(self.a, self.b)


def body_mask(dx, dy, bodies, ox=0.0, oy=0.0) -> np.ndarray:
    """uint8 cell mask, 1 where the cell centre lies inside a body."""
    xc, yc = centres(dx, ox), centres(dy, oy)
    X, Y = np.meshgrid(xc, yc)
    m = np.zeros(X.shape, dtype=bool)
    for bd in bodies:
        m |= bd.level(X, Y) < 0
    return m.astype(np.uint8)


def _smoothed_indicator(bodies, X, Y, h):
    chi = np.zeros_like(X)
    for bd in bodies:
        chi = np.maximum(chi, 0.5 * (1.0 - np.tanh(bd.level(X, Y) / (0.75 * h))))
    return chi


def mask_rhs(dx, dy, bodies, g: np.random.Generator, amp: float = 0.1,
             nmodes: int = 6, ox=0.0, oy=0.0, stream=(1.0, 0.0)):
    """Source ``S = D u*`` of an immersed-boundary projection step.

    ``u** = stream + amp * (random smooth field)`` lives on the staggered
    faces; ``u* = (1 - chi) u**`` with ``chi`` the body indicator smoothed
    over about 1.5 local cells (a stand-in for the regularised forcing of
    Eqs. 4-5).  ``D`` is the cell divergence.  The result is made compatible
    (zero volume-weighted mean).  The mask never enters the operator.
    """
    nx, ny = dx.size, dy.size
    lx, ly = dx.sum(), dy.sum()
    xf = ox + np.concatenate([[0.0], np.cumsum(dx)])
    yf = oy + np.concatenate([[0.0], np.cumsum(dy)])
    xc, yc = centres(dx, ox), centres(dy, oy)

    def field(X, Y):
        out = np.zeros_like(X)
        for _ in range(nmodes):
            kx, ky = g.integers(1, 6), g.integers(1, 6)
            p1, p2 = g.uniform(0, 2 * np.pi, 2)
            out += g.standard_normal() * np.sin(np.pi * kx * X / lx + p1) * np.sin(np.pi * ky * Y / ly + p2)
        return out / math.sqrt(nmodes)

    # u on x-faces: [ny, nx+1]; v on y-faces: [ny+1, nx]
    XU, YU = np.meshgrid(xf, yc)
    XV, YV = np.meshgrid(xc, yf)
    hu = np.sqrt(np.outer(dy, np.concatenate([[dx[0]], 0.5 * (dx[:-1] + dx[1:]), [dx[-1]]])))
    hv = np.sqrt(np.outer(np.concatenate([[dy[0]], 0.5 * (dy[:-1] + dy[1:]), [dy[-1]]]), dx))
    u = stream[0] + amp * field(XU, YU)
    v = stream[1] + amp * field(XV, YV)
    if bodies:
        u *= 1.0 - _smoothed_indicator(bodies, XU, YU, hu)
        v *= 1.0 - _smoothed_indicator(bodies, XV, YV, hv)
    div = (u[:, 1:] - u[:, :-1]) / dx[None, :] + (v[1:, :] - v[:-1, :]) / dy[:, None]
    return _zero_volume_mean(div, dx, dy)


# ---------------------------------------------------------------------------
# Random grid families and obstacles
# ---------------------------------------------------------------------------

def random_spacing(n: int, g: np.random.Generator, length: float = 1.0,
                   box_bias=None) -> np.ndarray:
    """One axis of a random stretched grid: tanh with ``beta ~ U(0.5, 2.5)``
    or a refined box (centre ``U(0.2, 0.8)``, width ``U(0.1, 0.4)``, growth
    ``U(1.02, 1.08)``), each with probability 1/2."""
    if (g.uniform() < 0.5 and box_bias is None) or n < 8:
        return tanh_spacing(n, g.uniform(0.5, 2.5), length) if n > 1 else np.full(1, length)
    c = g.uniform(0.2, 0.8) if box_bias is None else box_bias
    w = g.uniform(0.1, 0.4)
    a, b = max(0.02, c - w / 2), min(0.98, c + w / 2)
    return box_spacing(n, a * length, b * length, g.uniform(1.02, 1.08), length)


def random_bodies(g: np.random.Generator, max_bodies: int = 3):
    """0..max_bodies non-overlapping circles / ellipses, centres in [0.2, 0.8]^2."""
    k = int(g.integers(0, max_bodies + 1))
    out = []
    tries = 0
    while len(out) < k and tries < 200:
        tries += 1
        cx, cy = g.uniform(0.2, 0.8, 2)
        if g.uniform() < 0.5:
            r = 0.5 * g.uniform(0.05, 0.15)
            bd = Body(cx, cy, r, r)
        else:
            a = g.uniform(0.03, 0.1)
            bd = Body(cx, cy, a, a / g.uniform(1.0, 4.0), g.uniform(0, np.pi))
        if all(math.hypot(bd.cx - o.cx, bd.cy - o.cy) > max(bd.a, bd.b) + max(o.a, o.b) + 0.02 for o in out):
            out.append(bd)
    return out


# ---------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    dx: np.ndarray
    dy: np.ndarray
    f: np.ndarray                         # source S, [ny, nx]
    mask: np.ndarray | None = None        # uint8 [ny, nx] or None
    bodies: list = field(default_factory=list)
    tol: float = 1e-8

    @property
    def nx(self):
        return self.dx.size

    @property
    def ny(self):
        return self.dy.size


def config1(i: int = 0) -> Workload:
    """64x64, tanh stretching beta=2, 8 Gaussians (seed 1000 + i)."""
    g = rng(1000 + i)
    dx = tanh_spacing(64, 2.0)
    dy = tanh_spacing(64, 2.0)
    return Workload("tanh64_gauss8", dx, dy, gaussian_rhs(dx, dy, g))


def config2(i: int = 0, n: int = 512) -> Workload:
    """512x512 refined box [0.4, 0.6]^2 with growth 1.05, random Fourier
    source with 1/|k|^2 amplitudes up to |k| = 32 (seed 2000 + i)."""
    g = rng(2000 + i)
    dx = box_spacing(n, 0.4, 0.6, 1.05)
    dy = box_spacing(n, 0.4, 0.6, 1.05)
    return Workload(f"box{n}_fourier32", dx, dy, fourier_rhs(dx, dy, g))


def config3(i: int = 0, n: int = 256) -> Workload:
    """256x256 grid refined around a cylinder (D = 0.1 at (0.4, 0.5)); the
    source is the masked divergence of a perturbed stream (seed 3000 + i)."""
    g = rng(3000 + i)
    dx = box_spacing(n, 0.25, 0.55, 1.05)
    dy = box_spacing(n, 0.35, 0.65, 1.05)
    bodies = [Body(0.4, 0.5, 0.05, 0.05)]
    return Workload(f"cyl{n}_mask", dx, dy, mask_rhs(dx, dy, bodies, g),
                    body_mask(dx, dy, bodies), bodies)


def config4(count: int = 64, nmin: int = 128, nmax: int = 768,
            multiple: int = 16) -> list[Workload]:
    """``count`` independent systems, ``n ~ U{nmin..nmax}`` (rounded to a
    multiple of ``multiple``), per-system stretching and 0-3 obstacles
    (seed 4000 + i)."""
    out = []
    for i in range(count):
        g = rng(4000 + i)
        n = int(g.integers(nmin, nmax + 1))
        n = max(multiple, (n // multiple) * multiple)
        dx = random_spacing(n, g)
        dy = random_spacing(n, g)
        bodies = random_bodies(g)
        out.append(Workload(f"batch{i}_n{n}", dx, dy,
                            mask_rhs(dx, dy, bodies, g),
                            body_mask(dx, dy, bodies), bodies))
    return out


def config5_grid(nx: int = 2048, ny: int = 1024):
    """[0,2]x[0,1]; x refined over [0.4, 1.4] (body + wake), y over
    [0.4, 0.6]; growth 1.05; cylinder D = 0.1 at (0.5, 0.5)."""
    dx = box_spacing(nx, 0.4, 1.4, 1.05, 2.0)
    dy = box_spacing(ny, 0.4, 0.6, 1.05, 1.0)
    return dx, dy, [Body(0.5, 0.5, 0.05, 0.05)]


def _masked_indicator(bodies, xs, ys, hfun, reach=0.05):
    """chi on the tensor grid xs (columns) x ys (rows), evaluated only inside
    each body's bounding box widened by `reach` (zero elsewhere)."""
    chi = np.zeros((ys.size, xs.size))
    for bd in bodies:
        r = max(bd.a, bd.b) + reach
        i0, i1 = np.searchsorted(xs, bd.cx - r), np.searchsorted(xs, bd.cx + r)
        j0, j1 = np.searchsorted(ys, bd.cy - r), np.searchsorted(ys, bd.cy + r)
        if i1 <= i0 or j1 <= j0:
            continue
        X, Y = np.meshgrid(xs[i0:i1], ys[j0:j1])
        h = hfun(slice(j0, j1), slice(i0, i1))
        chi[j0:j1, i0:i1] = np.maximum(chi[j0:j1, i0:i1],
                                       0.5 * (1.0 - np.tanh(bd.level(X, Y) / (0.75 * h))))
    return chi


def config5_rhs(t: int, dx, dy, bodies, strouhal: float = 0.165,
                dt: float = 0.05) -> np.ndarray:
    """Time-sequence stand-in for the flow solver's PPE source at step ``t``:
    masked divergence of the intermediate velocity of ``config5_velocity``."""
    u, v = config5_velocity(t, dx, dy, bodies, strouhal, dt)
    div = (u[:, 1:] - u[:, :-1]) / dx[None, :] + (v[1:, :] - v[:-1, :]) / dy[:, None]
    return _zero_volume_mean(div, dx, dy)


def config5_velocity(t: int, dx, dy, bodies, strouhal: float = 0.165, dt: float = 0.05):
    """Stand-in for the intermediate velocity u* of step ``t`` (the momentum
    and immersed-boundary steps, Eqs. 3-5, are not part of this library): a
    uniform stream carrying a row of alternating Gaussian vortices advected
    downstream with Strouhal number 0.165, plus a small seeded perturbation
    (seed 5000 + t), masked by the smoothed body indicator.  Staggered faces:
    u [ny, nx+1], v [ny+1, nx]; the stream enters and leaves through the left
    and right walls with equal fluxes."""
    g = rng(5000 + t)
    lx = dx.sum()
    xf = np.concatenate([[0.0], np.cumsum(dx)])
    yf = np.concatenate([[0.0], np.cumsum(dy)])
    xc, yc = centres(dx), centres(dy)
    period = 0.1 / strouhal                  # D / (St U), U = 1
    time = t * dt
    sig = 0.03

    def vortex_uv(xs, ys):
        # separable Gaussians: u = -(y - py) e, v = (x - px) e, e = gam gx(x) gy(y)
        u = np.zeros((ys.size, xs.size))
        v = np.zeros((ys.size, xs.size))
        for k in range(12):
            age = (time + k * period / 2) % (6 * period)
            px = 0.6 + age
            if px > lx - 0.05:
                continue
            py = 0.5 + (0.04 if k % 2 else -0.04)
            gam = 0.3 * (1 if k % 2 else -1)
            gx = np.exp(-((xs - px) ** 2) / (2 * sig * sig))
            gy = np.exp(-((ys - py) ** 2) / (2 * sig * sig))
            u -= gam * np.outer(gy * (ys - py), gx)
            v += gam * np.outer(gy, gx * (xs - px))
        return u, v

    u = 1.0 + vortex_uv(xf, yc)[0] + 0.02 * g.standard_normal((yc.size, xf.size))
    v = vortex_uv(xc, yf)[1] + 0.02 * g.standard_normal((yf.size, xc.size))
    wx = np.concatenate([[dx[0]], 0.5 * (dx[:-1] + dx[1:]), [dx[-1]]])
    wy = np.concatenate([[dy[0]], 0.5 * (dy[:-1] + dy[1:]), [dy[-1]]])
    u *= 1.0 - _masked_indicator(bodies, xf, yc, lambda J, I_: np.sqrt(np.outer(dy[J], wx[I_])))
    v *= 1.0 - _masked_indicator(bodies, xc, yf, lambda J, I_: np.sqrt(np.outer(wy[J], dx[I_])))
    u[:, -1] = u[:, 0]                        # outflow = inflow: the walls' net flux vanishes
    v[0, :] = v[-1, :] = 0.0
    return u, v


def training_rhs(dx, dy, g: np.random.Generator) -> np.ndarray:
    """One fabricated training source: with probability 1/2 a sum of 4-16
    Gaussians (sigma in [0.01, 0.2]), else a 1/|k|^2 Fourier field with
    ``|k| <= 32``."""
    if g.uniform() < 0.5:
        return gaussian_rhs(dx, dy, g, int(g.integers(4, 17)), (0.01, 0.2))
    return fourier_rhs(dx, dy, g, 32)


# ---------------------------------------------------------------------------
# Network parameters (seeded initial values; shapes fix the layout)
# ---------------------------------------------------------------------------

@dataclass(frozen=True)
class NetConfig:
    """Grid-spacing-aware U-Net-branch DeepONet.

    ``widths[k]`` channels at U-Net level ``k`` (levels = len(widths));
    ``c_last`` branch/trunk feature count; ``trunk`` hidden widths of the
    coordinate MLP; ``phi_hidden`` width of each Mesh-Conv weight network.
    """
    widths: tuple = (32, 64, 128, 256)
    c_last: int = 100
    trunk: tuple = (100, 200)
    phi_hidden: int = 16
    mesh_conv: bool = True

    @property
    def levels(self):
        return len(self.widths)


def conv_layers(cfg: NetConfig):
    """Ordered list of (name, cin, cout, level) for every 3x3 Mesh-Conv."""
    w = cfg.widths
    L = cfg.levels
    out = []
    cin = 1
    for k in range(L):
        out.append((f"enc{k}a", cin, w[k], k))
        out.append((f"enc{k}b", w[k], w[k], k))
        cin = w[k]
    for k in range(L - 2, -1, -1):
        out.append((f"up{k}", w[k + 1], w[k], k))
        out.append((f"dec{k}a", 2 * w[k], w[k], k))
        out.append((f"dec{k}b", w[k], w[k], k))
    return out


def net_param_shapes(cfg: NetConfig):
    """Ordered ``name -> shape`` of every parameter (FP32)."""
    shapes = {}
    for name, ci, co, _ in conv_layers(cfg):
        shapes[f"{name}.w"] = (co, ci, 3, 3)
        shapes[f"{name}.b"] = (co,)
        shapes[f"{name}.phi1.w"] = (cfg.phi_hidden, 4)
        shapes[f"{name}.phi1.b"] = (cfg.phi_hidden,)
        shapes[f"{name}.phi2.w"] = (cfg.phi_hidden,)
        shapes[f"{name}.phi2.b"] = (1,)
    shapes["head.w"] = (cfg.c_last, cfg.widths[0])
    shapes["head.b"] = (cfg.c_last,)
    dims = (2,) + tuple(cfg.trunk) + (cfg.c_last,)
    for i in range(len(dims) - 1):
        shapes[f"trunk{i}.w"] = (dims[i + 1], dims[i])
        shapes[f"trunk{i}.b"] = (dims[i + 1],)
    shapes["out.b"] = (1,)
    return shapes


def net_params(cfg: NetConfig, seed: int, phi_scale: float = 0.1) -> dict:
    """Seeded initial parameters (He-normal convolutions, Glorot trunk,
    small weight-network parameters so that eta starts near 1)."""
    g = rng(seed)
    p = {}
    for name, shape in net_param_shapes(cfg).items():
        if name.endswith(".w") and ".phi" not in name and len(shape) == 4:
            fan_in = shape[1] * 9
            a = g.standard_normal(shape) * math.sqrt(2.0 / fan_in)
        elif ".phi" in name:
            a = g.standard_normal(shape) * phi_scale
        elif name.startswith("trunk") and name.endswith(".w"):
            a = g.standard_normal(shape) * math.sqrt(2.0 / (shape[0] + shape[1]))
        elif name == "head.w":
            a = g.standard_normal(shape) * math.sqrt(1.0 / shape[1])
        else:
            a = np.zeros(shape)
        p[name] = a.astype(np.float32)
    return p
