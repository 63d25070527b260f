"""The C-ABI library builds for sm_103a, loads, and exports every function
that ``include/*.h`` declares (no compute calls: this runs without a GPU)."""
import glob
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        names |= set(re.findall(r"PPE_API\s+[\w\s\*]+?\b(\w+)\s*\(", txt))
    return names


def test_header_declares_the_solver_calls():
    names = _declared()
    for n in ["ppe_create_grid", "ppe_destroy_grid", "ppe_solve", "ppe_solve_batch", "ppe_apply", "ppe_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2604_01800_gb300 import _lib, build
    path = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    missing = sorted(_declared() - exported)
    assert not missing, missing
    L = _lib.load(build_if_missing=False)
    for n in _declared():
        assert getattr(L, n) is not None
    assert b"sm_103a" in L.ppe_version()


def test_binding_covers_header():
    from paper_2604_01800_gb300 import _lib
    assert _declared() <= set(_lib.exported_names())


def test_struct_layouts_agree_with_the_header():
    """The host-only default fillers run without a GPU: each field the binding
    reads back must hold the value the header documents, which fails if the
    binding's struct layout drifts from the header's."""
    import ctypes

    from paper_2604_01800_gb300 import _lib
    L = _lib.load()
    o = _lib.ppe_solve_opts()
    L.ppe_default_options(ctypes.byref(o))
    assert (o.max_iters, o.num_cg, o.num_dlsm, o.hybrid_budget) == (200000, 3, 2, 20000)
    assert (o.inner_rtol, o.dlsm_guard) == (0.3, 1e-10)
    assert (o.blocks_per_sm, o.keep_dir_after_dlsm, o.iter_pass) == (2, 0, 0)
    assert (o.dlsm_stall_limit, o.dlsm_cost_iters) == (6, 16)
    assert (o.spin_limit_ms, o.host_loop, o.debug_skip_block, o.preconditioner) == (2000, 0, 0, 0)
    assert list(o.reserved) == [0] * len(o.reserved)
    c = _lib.ppe_net_config()
    L.net_default_config(ctypes.byref(c))
    assert c.levels == 4 and list(c.widths)[:4] == [32, 64, 128, 256] and c.c_last == 100
    assert list(c.trunk_hidden) == [100, 200] and (c.phi_hidden, c.mesh_conv) == (16, 1)
    h = _lib.ppe_train_hparams()
    L.net_default_hparams(ctypes.byref(h))
    assert (h.lr0, h.total_steps, h.rho, h.beta1, h.beta2, h.eps) == (2e-4, 1000000, 2e-4, 0.9, 0.999, 1e-8)
