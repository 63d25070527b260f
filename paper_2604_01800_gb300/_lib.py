"""ctypes binding of ``include/ppe.h`` (argument marshalling only).

Every computation runs inside ``lib/libppe_gb300.so``.  Loading fails loudly
when the library has not been built: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

_lib = None

PPE_OK, PPE_ERR_ARG, PPE_ERR_CUDA, PPE_ERR_NOMEM, PPE_ERR_INCOMPATIBLE_RHS = 0, 1, 2, 3, 4
PPE_ERR_NOT_CONVERGED, PPE_ERR_TIMEOUT, PPE_ERR_NAN, PPE_ERR_NO_NET, PPE_ERR_FORMAT = 5, 6, 7, 8, 9
PPE_MODE_PCG, PPE_MODE_HYBRID = 0, 1
PPE_PRECOND_JACOBI, PPE_PRECOND_MG = 0, 1
PPE_PREC_FP64, PPE_PREC_MIXED = 0, 1
PPE_BC_NEUMANN = 0

STATUS_NAMES = {0: "PPE_OK", 1: "PPE_ERR_ARG", 2: "PPE_ERR_CUDA", 3: "PPE_ERR_NOMEM",
                4: "PPE_ERR_INCOMPATIBLE_RHS", 5: "PPE_ERR_NOT_CONVERGED", 6: "PPE_ERR_TIMEOUT",
                7: "PPE_ERR_NAN", 8: "PPE_ERR_NO_NET", 9: "PPE_ERR_FORMAT"}


class ppe_solve_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iters_pcg", ctypes.c_int32), ("iters_dlsm", ctypes.c_int32),
                ("dlsm_skipped", ctypes.c_int32), ("refinements", ctypes.c_int32), ("fell_back", ctypes.c_int32),
                ("net_calls", ctypes.c_int32), ("launches", ctypes.c_int32), ("rel_res_true", ctypes.c_double),
                ("incompat", ctypes.c_double), ("ms_total", ctypes.c_double), ("ms_net", ctypes.c_double),
                ("ms_pcg", ctypes.c_double), ("ms_dlsm", ctypes.c_double), ("ms_refine", ctypes.c_double),
                ("drive", ctypes.c_int32), ("precision_fallback", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ppe_solve_opts(ctypes.Structure):
    _fields_ = [("max_iters", ctypes.c_int32), ("num_cg", ctypes.c_int32), ("num_dlsm", ctypes.c_int32),
                ("hybrid_budget", ctypes.c_int32), ("inner_rtol", ctypes.c_double), ("dlsm_guard", ctypes.c_double),
                ("blocks_per_sm", ctypes.c_int32), ("keep_dir_after_dlsm", ctypes.c_int32),
                ("iter_pass", ctypes.c_int32), ("dlsm_stall_limit", ctypes.c_int32),
                ("dlsm_cost_iters", ctypes.c_int32), ("spin_limit_ms", ctypes.c_int32), ("host_loop", ctypes.c_int32),
                ("debug_skip_block", ctypes.c_int32), ("preconditioner", ctypes.c_int32),
                ("debug_force_stall", ctypes.c_int32), ("tile_rows", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 2)]


class ppe_tune_report(ctypes.Structure):
    _fields_ = [("iter_pass", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("us_per_iter", ctypes.c_double * 3), ("tile_rows", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]


class ppe_net_config(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int32), ("widths", ctypes.c_int32 * 6), ("c_last", ctypes.c_int32),
                ("trunk_hidden", ctypes.c_int32 * 2), ("phi_hidden", ctypes.c_int32), ("mesh_conv", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 4)]


# void (*)(void *user, const float *r_hat, float *e, int nx, int ny, void *stream)
ppe_direction_fn = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                    ctypes.c_int, ctypes.c_void_p)


class ppe_train_hparams(ctypes.Structure):
    _fields_ = [("lr0", ctypes.c_double), ("total_steps", ctypes.c_int64), ("rho", ctypes.c_double),
                ("beta1", ctypes.c_double), ("beta2", ctypes.c_double), ("eps", ctypes.c_double),
                ("reserved", ctypes.c_int32 * 8)]


class PPEError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


# (name, restype, argtypes) of every exported symbol
_P = ctypes.c_void_p
_SIGS = [
    ("ppe_default_options", None, [ctypes.POINTER(ppe_solve_opts)]),
    ("ppe_create_grid", ctypes.c_int, [ctypes.c_int, ctypes.c_int, _P, _P, ctypes.c_int, _P, ctypes.POINTER(_P)]),
    ("ppe_destroy_grid", None, [_P]),
    ("ppe_grid_shape", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    ("ppe_set_options", ctypes.c_int, [_P, ctypes.POINTER(ppe_solve_opts)]),
    ("ppe_apply", ctypes.c_int, [_P, _P, _P, _P]),
    ("ppe_residual", ctypes.c_int, [_P, _P, _P, _P, _P]),
    ("ppe_solve", ctypes.c_int, [_P, _P, _P, ctypes.c_double, ctypes.c_int, ctypes.c_int, _P, _P,
                                 ctypes.POINTER(ppe_solve_info)]),
    ("ppe_solve_batch", ctypes.c_int, [ctypes.c_int, _P, _P, _P, ctypes.c_double, ctypes.c_int, ctypes.c_int, _P,
                                       _P, ctypes.POINTER(ppe_solve_info)]),
    ("net_default_config", None, [ctypes.POINTER(ppe_net_config)]),
    ("net_create", ctypes.c_int, [ctypes.POINTER(ppe_net_config), ctypes.c_uint64, ctypes.POINTER(_P)]),
    ("net_destroy", None, [_P]),
    ("net_param_count", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64)]),
    ("net_get_config", ctypes.c_int, [_P, ctypes.POINTER(ppe_net_config)]),
    ("net_set_params", ctypes.c_int, [_P, _P, ctypes.c_int64]),
    ("net_get_params", ctypes.c_int, [_P, _P, ctypes.c_int64]),
    ("net_save", ctypes.c_int, [_P, ctypes.c_char_p]),
    ("net_save_params", ctypes.c_int, [_P, ctypes.c_char_p]),
    ("net_load", ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(_P)]),
    ("net_attach", ctypes.c_int, [_P, _P]),
    ("net_infer", ctypes.c_int, [_P, _P, _P, _P, _P]),
    ("net_infer_batch", ctypes.c_int, [_P, _P, ctypes.c_int, _P, _P, _P]),
    ("ppe_debug_conv3x3", ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, _P, ctypes.c_int, _P]),
    ("ppe_set_direction_source", ctypes.c_int, [_P, _P, _P]),
    ("net_default_hparams", None, [ctypes.POINTER(ppe_train_hparams)]),
    ("net_train_step", ctypes.c_int, [_P, _P, ctypes.c_int, _P, ctypes.POINTER(ppe_train_hparams), _P,
                                      ctypes.POINTER(ctypes.c_double)]),
    ("net_loss_grad", ctypes.c_int, [_P, _P, ctypes.c_int, _P, _P, ctypes.POINTER(ctypes.c_double), _P]),
    ("net_get_step", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64)]),
    ("ppe_solve_noalloc", ctypes.c_int, [ctypes.c_int, ctypes.c_int, _P, _P, _P, _P, ctypes.c_double, ctypes.c_int,
                                         _P, ctypes.POINTER(ppe_solve_info)]),
    ("ppe_autotune", ctypes.c_int, [_P, _P, ctypes.POINTER(ppe_tune_report)]),
    ("ppe_debug_mg_vcycle", ctypes.c_int, [_P, _P, _P, _P]),
    ("ppe_debug_wgrad", ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P,
                                       ctypes.c_int, _P]),
    ("ppe_debug_pick_variant", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              _P, _P]),
    ("ppe_debug_plan_ranges", ctypes.c_int, [ctypes.c_int, _P, ctypes.c_int, ctypes.c_int, _P, _P, _P, _P, _P, _P,
                                             _P]),
    ("ppe_debug_gemm", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, ctypes.c_int, ctypes.c_int, _P,
                                      ctypes.c_int, ctypes.c_int, _P, ctypes.c_int, _P, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_int, _P, _P]),
    ("ppe_source", ctypes.c_int, [_P, _P, _P, ctypes.c_double, _P, _P]),
    ("ppe_project", ctypes.c_int, [_P, _P, ctypes.c_double, _P, _P, _P, _P]),
    ("ppe_last_error", ctypes.c_char_p, []),
    ("ppe_version", ctypes.c_char_p, []),
]


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load the CUDA library (building it first if allowed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    L = ctypes.CDLL(path)
    for name, res, args in _SIGS:
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def exported_names():
    return [s[0] for s in _SIGS]


def check(status: int, what: str = ""):
    if status != PPE_OK:
        msg = load().ppe_last_error().decode(errors="replace")
        raise PPEError(status, f"{what}: {msg}" if what else msg)
