"""Parity of the network's CUDA path with the FP64 network oracle.

Tolerances come from the arithmetic: activations and weights are rounded to
BF16 (relative rounding 2^-9) at every layer and products accumulate in FP32.
* One convolution on BF16-exact inputs: the oracle evaluates the same
  products in FP64, so the only differences are FP32 accumulation order and
  rounding: |err| <= 1e-5 * sum |w x| per output.
* A whole forward pass compounds ~2^-9 per layer over the network's depth;
  the test bound on the relative L2 error of e is 3e-2 and of each sample's
  direction (cosine) 0.999.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import net_oracle as N  # noqa: E402
from paper_2604_01800_gb300 import inputs as I  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_01800_gb300 import api as A
    return A


def bf16_round(a):
    return torch.tensor(np.asarray(a, np.float32)).to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64)


def _conv_case(api, B, H, W, cin, cout, impl, seed):
    g = I.rng(seed)
    x = bf16_round(g.standard_normal((B, H, W, cin)))
    w = bf16_round(g.standard_normal((cout, 9, cin)) / np.sqrt(9 * cin))
    b = g.standard_normal(cout).astype(np.float32)
    dx = torch.tensor(x, dtype=torch.bfloat16, device="cuda")
    dw = torch.tensor(w, dtype=torch.bfloat16, device="cuda")
    db = torch.tensor(b, dtype=torch.float32, device="cuda")
    out = torch.zeros(B, H, W, cout, dtype=torch.float32, device="cuda")
    import ctypes
    L = api._lib.load()
    st = L.ppe_debug_conv3x3(ctypes.c_void_p(dx.data_ptr()), ctypes.c_void_p(dw.data_ptr()),
                             ctypes.c_void_p(db.data_ptr()), B, H, W, cin, cout, ctypes.c_void_p(out.data_ptr()),
                             impl, None)
    api._lib.check(st, "ppe_debug_conv3x3")
    torch.cuda.synchronize()
    # oracle: W[co][ci][ky][kx] from the packed [co][tap][ci]
    Wt = w.reshape(cout, 3, 3, cin).transpose(0, 3, 1, 2)
    ref = N.conv3x3(x.transpose(0, 3, 1, 2), Wt, b.astype(np.float64)).transpose(0, 2, 3, 1)
    scale = N.conv3x3(np.abs(x).transpose(0, 3, 1, 2), np.abs(Wt), np.abs(b.astype(np.float64))).transpose(0, 2, 3, 1)
    err = np.abs(out.cpu().numpy() - ref)
    assert np.all(err <= 1e-5 * scale + 1e-6), float((err / (scale + 1e-30)).max())


# The last two shapes have far more output tiles (of 128 pixels) than the
# kernel has CTAs (one or two per SM): 1,024 and 512 tiles, so every CTA walks
# several tiles, alternating its two TMEM accumulators and carrying the stage
# ring's phases from tile to tile, as at the full 256^2 and 512^2 sizes.  They
# cover both channel-block widths of the kernel (32- and 64-channel blocks).
@pytest.mark.parametrize("B,H,W,cin,cout", [(1, 16, 16, 16, 16), (2, 13, 21, 32, 48), (1, 8, 40, 64, 32),
                                             (1, 32, 32, 256, 128), (2, 64, 64, 64, 256), (1, 7, 9, 16, 16),
                                             (3, 24, 40, 128, 64), (1, 256, 8, 32, 32), (2, 256, 256, 32, 32),
                                             (1, 256, 256, 64, 64)])
@pytest.mark.parametrize("impl", [0, 1], ids=["tcgen05", "simt"])
def test_conv_matches_oracle(api, B, H, W, cin, cout, impl):
    _conv_case(api, B, H, W, cin, cout, impl, 100 + H)


def _tiny_cfg():
    return I.NetConfig(widths=(16, 32), c_last=8, trunk=(16, 24), phi_hidden=4)


def _make_net(api, cfg, seed, phi_scale=0.5):
    P = I.net_params(cfg, seed, phi_scale=phi_scale)
    g = I.rng(seed + 7)
    for k in P:
        if k.endswith(".b"):
            P[k] = (0.1 * g.standard_normal(P[k].shape)).astype(np.float32)
    c = api.net_default_config(widths=list(cfg.widths), c_last=cfg.c_last, trunk_hidden=list(cfg.trunk),
                               phi_hidden=cfg.phi_hidden, mesh_conv=int(cfg.mesh_conv))
    net = api.net_create(c, 1)
    flat = api.flatten_params(P, cfg)
    assert flat.size == net.param_count
    net.set_params(flat)
    return net, P


# "conv": the standard-convolution ablation of Sec. 3 (mesh_conv = 0, eta = 1
# in every layer), against the oracle's forward with the same switch.
@pytest.mark.parametrize("cfgname,nx,ny,B", [("tiny", 29, 21, 2), ("tiny", 32, 32, 1), ("full", 64, 48, 1),
                                             ("full", 50, 70, 2), ("conv", 29, 21, 2), ("fullconv", 64, 48, 1)])
def test_forward_matches_oracle(api, cfgname, nx, ny, B):
    cfg = {"tiny": _tiny_cfg(), "full": I.NetConfig(),
           "conv": I.NetConfig(widths=(16, 32), c_last=8, trunk=(16, 24), phi_hidden=4, mesh_conv=False),
           "fullconv": I.NetConfig(mesh_conv=False)}[cfgname]
    net, P = _make_net(api, cfg, 3)
    g = I.rng(11)
    dx, dy = I.random_spacing(nx, g), I.random_spacing(ny, g)
    R = g.standard_normal((B, ny, nx)).astype(np.float32)
    grid = api.ppe_create_grid(dx, dy)
    net.attach(grid)
    r = torch.tensor(R, dtype=torch.float32, device="cuda")
    e = torch.zeros_like(r)
    net.infer(grid, r, e)
    torch.cuda.synchronize()
    geo = N.Geometry(dx, dy, cfg.levels)
    eo, _ = N.forward(P, geo, R.astype(np.float64), cfg.widths, cfg.mesh_conv, len(cfg.trunk) + 1)
    eg = e.cpu().numpy().astype(np.float64)
    rel = np.linalg.norm(eg - eo) / np.linalg.norm(eo)
    assert rel <= 3e-2, rel
    for b in range(B):
        cos = (eg[b] * eo[b]).sum() / np.linalg.norm(eg[b]) / np.linalg.norm(eo[b])
        assert cos >= 0.999, cos


def test_weights_file_roundtrip(api, tmp_path):
    cfg = _tiny_cfg()
    net, P = _make_net(api, cfg, 5)
    path = str(tmp_path / "w.ppenet")
    net.save(path)
    net2 = api.net_load(path)
    assert np.array_equal(net2.get_params(), net.get_params())
    assert net2.step == net.step
    raw = bytearray(open(path, "rb").read())
    raw[100] ^= 0xFF
    bad = tmp_path / "bad.ppenet"
    bad.write_bytes(bytes(raw))
    with pytest.raises(api.PPEError) as ei:
        api.net_load(str(bad))
    assert ei.value.status == api._lib.PPE_ERR_FORMAT


def test_forward_full_config_on_cylinder_grid(api):
    """The full 32-256 network on the 256^2 cylinder grid: every layer runs at
    its full size (the 256^2 layers walk several tiles per CTA), checked
    element by element against the oracle's forward pass."""
    cfg = I.NetConfig()
    net, P = _make_net(api, cfg, 3)
    w = I.config3(0)
    g = I.rng(19)
    R = g.standard_normal((1, w.ny, w.nx)).astype(np.float32)
    grid = api.ppe_create_grid(w.dx, w.dy)
    net.attach(grid)
    r = torch.tensor(R, dtype=torch.float32, device="cuda")
    e = torch.zeros_like(r)
    net.infer(grid, r, e)
    torch.cuda.synchronize()
    geo = N.Geometry(w.dx, w.dy, cfg.levels)
    eo, _ = N.forward(P, geo, R.astype(np.float64), cfg.widths, cfg.mesh_conv, len(cfg.trunk) + 1)
    eg = e.cpu().numpy().astype(np.float64)
    rel = np.linalg.norm(eg - eo) / np.linalg.norm(eo)
    cos = (eg * eo).sum() / np.linalg.norm(eg) / np.linalg.norm(eo)
    assert rel <= 3e-2 and cos >= 0.999, (rel, cos)
