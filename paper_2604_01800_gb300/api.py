"""Python face of the C ABI: same names as ``include/ppe.h``.

Each function only marshals arguments (torch CUDA tensors -> device
pointers, the current torch stream -> ``cudaStream_t``) and calls into the
CUDA library.  PyTorch supplies device memory and streams; nothing here
computes.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import (PPE_MODE_HYBRID, PPE_MODE_PCG, PPE_PREC_FP64, PPE_PREC_MIXED, PPEError, check,
                   ppe_solve_info, ppe_solve_opts)

__all__ = ["Net", "net_create", "net_load", "net_default_config", "Grid", "ppe_create_grid", "ppe_destroy_grid", "ppe_apply", "ppe_solve", "ppe_solve_batch",
           "ppe_set_options", "ppe_default_options", "ppe_set_direction_source", "ppe_residual", "PPE_MODE_PCG", "PPE_MODE_HYBRID", "PPE_PREC_FP64",
           "PPE_PREC_MIXED", "PPEError"]


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _dptr(t: torch.Tensor, dtype=torch.float64, numel=None):
    if not (t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise ValueError(f"expected a contiguous CUDA {dtype} tensor")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"expected {numel} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


class Grid:
    """Owning wrapper of a ``ppe_grid*``."""

    def __init__(self, handle, nx, ny):
        self.handle = handle
        self.nx, self.ny = nx, ny

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def close(self):
        if self.handle:
            _lib.load().ppe_destroy_grid(self.handle)
            self.handle = None

    @property
    def shape(self):
        return (self.ny, self.nx)


def ppe_create_grid(dx, dy, mask=None, bc: int = 0) -> Grid:
    L = _lib.load()
    dx = np.ascontiguousarray(dx, dtype=np.float64)
    dy = np.ascontiguousarray(dy, dtype=np.float64)
    mptr = None
    if mask is not None:
        mask = np.ascontiguousarray(mask, dtype=np.uint8)
        mptr = mask.ctypes.data_as(ctypes.c_void_p)
    h = ctypes.c_void_p()
    st = L.ppe_create_grid(dx.size, dy.size, dx.ctypes.data_as(ctypes.c_void_p), dy.ctypes.data_as(ctypes.c_void_p),
                           bc, mptr, ctypes.byref(h))
    check(st, "ppe_create_grid")
    return Grid(h, dx.size, dy.size)


def ppe_destroy_grid(grid: Grid):
    grid.close()


def ppe_default_options() -> ppe_solve_opts:
    o = ppe_solve_opts()
    _lib.load().ppe_default_options(ctypes.byref(o))
    return o


def ppe_set_options(grid: Grid, opts: ppe_solve_opts | None = None, **kw):
    o = opts if opts is not None else ppe_default_options()
    for k, v in kw.items():
        setattr(o, k, v)
    check(_lib.load().ppe_set_options(grid.handle, ctypes.byref(o)), "ppe_set_options")
    return o


def ppe_autotune(grid: Grid, stream=None) -> dict:
    """Time the iteration-pass variants on this grid (mixed precision) and keep
    the fastest for later solves of this grid shape; returns the report."""
    rep = _lib.ppe_tune_report()
    check(_lib.load().ppe_autotune(grid.handle, _stream(stream), ctypes.byref(rep)), "ppe_autotune")
    return {"iter_pass": rep.iter_pass, "blocks_per_sm": rep.blocks_per_sm, "tile_rows": rep.tile_rows,
            "us_per_iter": {"tile": rep.us_per_iter[0], "stream": rep.us_per_iter[2]}}


def ppe_set_direction_source(grid: Grid, fn):
    """Install ``fn(r_hat, e, stream)`` (torch CUDA float32 tensors [ny, nx]
    viewing the library's staging buffers) as the DLSM direction source of
    ``grid``; ``None`` removes it."""
    if fn is None:
        grid._dir_cb = None
        check(_lib.load().ppe_set_direction_source(grid.handle, None, None), "ppe_set_direction_source")
        return

    def tramp(user, r_ptr, e_ptr, nx, ny, stream_ptr):
        n = nx * ny
        r = _wrap_device(r_ptr, n).view(ny, nx)
        e = _wrap_device(e_ptr, n).view(ny, nx)
        fn(r, e, stream_ptr)

    cb = _lib.ppe_direction_fn(tramp)
    grid._dir_cb = cb                       # keep the trampoline alive
    check(_lib.load().ppe_set_direction_source(grid.handle, ctypes.cast(cb, ctypes.c_void_p), None),
          "ppe_set_direction_source")


def _wrap_device(ptr, n):
    """A float32 CUDA tensor viewing n elements at device address ptr."""
    class _Iface:
        __cuda_array_interface__ = {"shape": (n,), "typestr": "<f4", "data": (int(ptr), False), "version": 2}
    return torch.as_tensor(_Iface(), device="cuda")


def ppe_apply(grid: Grid, x: torch.Tensor, y: torch.Tensor, stream=None):
    n = grid.nx * grid.ny
    check(_lib.load().ppe_apply(grid.handle, _dptr(x, numel=n), _dptr(y, numel=n), _stream(stream)), "ppe_apply")
    return y


def ppe_residual(grid: Grid, S: torch.Tensor, x: torch.Tensor, r: torch.Tensor, stream=None):
    """r = -V S - A x (FP64 device tensors [ny, nx])."""
    n = grid.nx * grid.ny
    check(_lib.load().ppe_residual(grid.handle, _dptr(S, numel=n), _dptr(x, numel=n), _dptr(r, numel=n),
                                   _stream(stream)), "ppe_residual")
    return r


def ppe_source(grid: Grid, u: torch.Tensor, v: torch.Tensor, dt: float, S: torch.Tensor, stream=None):
    """S = (D u* - bc2) / dt from the staggered faces u [ny, nx+1], v [ny+1, nx] (Eq. 6)."""
    nx, ny = grid.nx, grid.ny
    check(_lib.load().ppe_source(grid.handle, _dptr(u, numel=ny * (nx + 1)), _dptr(v, numel=(ny + 1) * nx),
                                 float(dt), _dptr(S, numel=nx * ny), _stream(stream)), "ppe_source")
    return S


def ppe_project(grid: Grid, dp: torch.Tensor, dt: float, u: torch.Tensor, v: torch.Tensor, p=None, stream=None):
    """u, v <- u, v - dt G dp on the interior faces (Eq. 7); p <- p + dp (Eq. 8)."""
    nx, ny = grid.nx, grid.ny
    pp = None if p is None else _dptr(p, numel=nx * ny)
    check(_lib.load().ppe_project(grid.handle, _dptr(dp, numel=nx * ny), float(dt), _dptr(u, numel=ny * (nx + 1)),
                                  _dptr(v, numel=(ny + 1) * nx), pp, _stream(stream)), "ppe_project")


def ppe_solve(grid: Grid, rhs: torch.Tensor, x: torch.Tensor, tol_rel: float = 1e-8, mode: int = PPE_MODE_PCG,
              precision: int = PPE_PREC_MIXED, net=None, stream=None, raise_on_error: bool = True) -> dict:
    """Solve M x = rhs in place of ``x``; returns the info report as a dict."""
    n = grid.nx * grid.ny
    info = ppe_solve_info()
    nh = None if net is None else net.handle
    st = _lib.load().ppe_solve(grid.handle, _dptr(rhs, numel=n), _dptr(x, numel=n), float(tol_rel), int(mode),
                               int(precision), nh, _stream(stream), ctypes.byref(info))
    d = info.as_dict()
    d["status"] = st
    if raise_on_error and st != _lib.PPE_OK:
        check(st, "ppe_solve")
    return d


def ppe_solve_batch(grids, rhs, xs, tol_rel: float = 1e-8, mode: int = PPE_MODE_PCG,
                    precision: int = PPE_PREC_MIXED, net=None, stream=None, raise_on_error: bool = True):
    n = len(grids)
    G = (ctypes.c_void_p * n)(*[g.handle for g in grids])
    R = (ctypes.c_void_p * n)(*[_dptr(r, numel=g.nx * g.ny).value for r, g in zip(rhs, grids)])
    X = (ctypes.c_void_p * n)(*[_dptr(x, numel=g.nx * g.ny).value for x, g in zip(xs, grids)])
    infos = (ppe_solve_info * n)()
    nh = None if net is None else net.handle
    st = _lib.load().ppe_solve_batch(n, ctypes.cast(G, ctypes.c_void_p), ctypes.cast(R, ctypes.c_void_p),
                                     ctypes.cast(X, ctypes.c_void_p), float(tol_rel), int(mode), int(precision), nh,
                                     _stream(stream), infos)
    if raise_on_error and st != _lib.PPE_OK:
        check(st, "ppe_solve_batch")
    return [i.as_dict() for i in infos], st


# ---------------------------------------------------------------------------
# network
# ---------------------------------------------------------------------------

def net_default_config(**kw) -> _lib.ppe_net_config:
    c = _lib.ppe_net_config()
    _lib.load().net_default_config(ctypes.byref(c))
    for k, v in kw.items():
        if k == "widths":
            c.levels = len(v)
            for i in range(6):
                c.widths[i] = v[i] if i < len(v) else 0
        elif k == "trunk_hidden":
            c.trunk_hidden[0], c.trunk_hidden[1] = v
        else:
            setattr(c, k, v)
    return c


class Net:
    """Owning wrapper of a ``ppe_net*``."""

    def __init__(self, handle):
        self.handle = handle

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def close(self):
        if self.handle:
            _lib.load().net_destroy(self.handle)
            self.handle = None

    @property
    def param_count(self) -> int:
        n = ctypes.c_int64()
        check(_lib.load().net_param_count(self.handle, ctypes.byref(n)), "net_param_count")
        return n.value

    def config(self) -> _lib.ppe_net_config:
        c = _lib.ppe_net_config()
        check(_lib.load().net_get_config(self.handle, ctypes.byref(c)), "net_get_config")
        return c

    def set_params(self, flat: np.ndarray):
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        check(_lib.load().net_set_params(self.handle, flat.ctypes.data_as(ctypes.c_void_p), flat.size), "net_set_params")

    def get_params(self) -> np.ndarray:
        out = np.empty(self.param_count, dtype=np.float32)
        check(_lib.load().net_get_params(self.handle, out.ctypes.data_as(ctypes.c_void_p), out.size), "net_get_params")
        return out

    def save(self, path: str, with_moments: bool = True):
        fn = _lib.load().net_save if with_moments else _lib.load().net_save_params
        check(fn(self.handle, path.encode()), "net_save")

    def attach(self, grid: Grid):
        check(_lib.load().net_attach(self.handle, grid.handle), "net_attach")

    def train_step(self, grid: Grid, R: torch.Tensor, hp=None, stream=None, **kw) -> float:
        """One SAM + Adam step on the batch R [B, ny, nx] (float32, CUDA)."""
        hp = hp if hp is not None else net_default_hparams(**kw)
        n = grid.nx * grid.ny
        b = R.numel() // n
        loss = ctypes.c_double()
        check(_lib.load().net_train_step(self.handle, grid.handle, b, _dptr(R, torch.float32, b * n), ctypes.byref(hp),
                                         _stream(stream), ctypes.byref(loss)), "net_train_step")
        return loss.value

    def loss_grad(self, grid: Grid, R: torch.Tensor, stream=None):
        """(loss, flat gradient) at the current parameters."""
        n = grid.nx * grid.ny
        b = R.numel() // n
        loss = ctypes.c_double()
        g = np.empty(self.param_count, dtype=np.float32)
        check(_lib.load().net_loss_grad(self.handle, grid.handle, b, _dptr(R, torch.float32, b * n), _stream(stream),
                                        ctypes.byref(loss), g.ctypes.data_as(ctypes.c_void_p)), "net_loss_grad")
        return loss.value, g

    @property
    def step(self) -> int:
        t = ctypes.c_int64()
        check(_lib.load().net_get_step(self.handle, ctypes.byref(t)), "net_get_step")
        return t.value

    def infer(self, grid: Grid, r: torch.Tensor, e: torch.Tensor, stream=None):
        n = grid.nx * grid.ny
        b = r.numel() // n
        check(_lib.load().net_infer_batch(self.handle, grid.handle, b, _dptr(r, torch.float32, b * n),
                                          _dptr(e, torch.float32, b * n), _stream(stream)), "net_infer")
        return e


def net_default_hparams(**kw) -> _lib.ppe_train_hparams:
    hp = _lib.ppe_train_hparams()
    _lib.load().net_default_hparams(ctypes.byref(hp))
    for k, v in kw.items():
        setattr(hp, k, v)
    return hp


def net_create(cfg=None, seed: int = 0) -> Net:
    cfg = cfg if cfg is not None else net_default_config()
    h = ctypes.c_void_p()
    check(_lib.load().net_create(ctypes.byref(cfg), seed, ctypes.byref(h)), "net_create")
    return Net(h)


def net_load(path: str) -> Net:
    h = ctypes.c_void_p()
    check(_lib.load().net_load(path.encode(), ctypes.byref(h)), "net_load")
    return Net(h)


def flatten_params(P: dict, cfg) -> np.ndarray:
    """Flatten a name -> array dict in the library's parameter order."""
    from .inputs import net_param_shapes
    return np.concatenate([np.asarray(P[k], np.float32).reshape(-1) for k in net_param_shapes(cfg)])


def unflatten_params(flat: np.ndarray, cfg) -> dict:
    """Inverse of flatten_params."""
    from .inputs import net_param_shapes
    out, off = {}, 0
    for k, shp in net_param_shapes(cfg).items():
        n = int(np.prod(shp))
        out[k] = flat[off:off + n].reshape(shp)
        off += n
    return out
