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
