"""ctypes declarations of the C ABI in include/dc.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libdc.so")

DC_OK = 0
STATUS_NAMES = {0: "DC_OK", 1: "DC_ERR_INVALID", 2: "DC_ERR_CUDA", 3: "DC_ERR_NOT_SPD", 4: "DC_ERR_OOM",
                5: "DC_ERR_NONFINITE", 6: "DC_ERR_NONCONVERGED", 7: "DC_ERR_STATE", 8: "DC_ERR_TIMEOUT"}
COMPLIANCE = {"rowsum": 0, "diag_pinv": 1, "diag_p": 2, "mass": 3}
LAYOUTS = {"node_major": 0, "component_major": 1}
DC_PLANE, DC_SPHERE, DC_CAPSULE, DC_MESH = 0, 1, 2, 3
DC_MAX_OBSTACLES = 16


class dc_obstacle(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("pad_", ctypes.c_int32), ("p", ctypes.c_double * 7)]


class dc_params(ctypes.Structure):
    _fields_ = [("k_stretch", ctypes.c_double), ("k_bend", ctypes.c_double), ("density", ctypes.c_double),
                ("mu", ctypes.c_double), ("h", ctypes.c_double), ("gravity", ctypes.c_double * 3),
                ("contact_margin", ctypes.c_double), ("adj_tol", ctypes.c_double),
                ("n_pd_iters", ctypes.c_int32), ("adj_max_iters", ctypes.c_int32),
                ("adj_restart", ctypes.c_int32), ("checkpoint_every", ctypes.c_int32),
                ("n_obstacles", ctypes.c_int32), ("adj_precond", ctypes.c_int32),
                ("global_solver", ctypes.c_int32), ("contact_compliance", ctypes.c_int32),
                ("adj_fallback", ctypes.c_int32), ("factor_on_gpu", ctypes.c_int32),
                ("obstacles", dc_obstacle * DC_MAX_OBSTACLES)]


class dc_stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("contacts_takeoff", ctypes.c_int64),
                ("contacts_stick", ctypes.c_int64), ("contacts_slip", ctypes.c_int64),
                ("adj_steps", ctypes.c_int64), ("adj_iters", ctypes.c_int64),
                ("adj_max_iters_seen", ctypes.c_int64), ("adj_nonconverged", ctypes.c_int64),
                ("adj_last_residual", ctypes.c_double), ("factor_nnz", ctypes.c_int64),
                ("solve_nnz", ctypes.c_int64), ("n_free", ctypes.c_int32), ("nd_levels", ctypes.c_int32),
                ("kernel_launches", ctypes.c_int64), ("timer_ms", ctypes.c_double),
                ("timer_launches", ctypes.c_int64), ("fwd_solve_nnz", ctypes.c_int64),
                ("bwd_solve_nnz", ctypes.c_int64), ("front_flops", ctypes.c_double),
                ("front_levels", ctypes.c_int32), ("n_supernodes", ctypes.c_int32),
                ("factorisations", ctypes.c_int64), ("n_instances", ctypes.c_int32), ("graphs", ctypes.c_int32),
                ("graph_replays", ctypes.c_int64), ("block_local", ctypes.c_int32), ("block_gather", ctypes.c_int32),
                ("block_node", ctypes.c_int32), ("block_elem", ctypes.c_int32), ("adj_batch_iters", ctypes.c_int64),
                ("global_solver", ctypes.c_int32), ("reserved_", ctypes.c_int32), ("psolve_flops", ctypes.c_double),
                ("adj_fallbacks", ctypes.c_int64), ("adj_fallback_iters", ctypes.c_int64),
                ("layout", ctypes.c_int32), ("contact_compliance", ctypes.c_int32),
                ("device_bytes", ctypes.c_int64), ("device_bytes_peak", ctypes.c_int64),
                ("n_nodes", ctypes.c_int32), ("n_tris", ctypes.c_int32), ("bend_nnz", ctypes.c_int64),
                ("front_entries", ctypes.c_int64)]


class dc_instance(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int32), ("n_tris", ctypes.c_int32), ("n_pins", ctypes.c_int32),
                ("pad_", ctypes.c_int32), ("rest_pos", ctypes.c_void_p), ("tris", ctypes.c_void_p),
                ("pins", ctypes.c_void_p)]

class dc_server_config(ctypes.Structure):
    _fields_ = [("n_slots", ctypes.c_int32), ("n_prep_threads", ctypes.c_int32), ("hbm_budget_bytes", ctypes.c_int64),
                ("max_prepared", ctypes.c_int32), ("device", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("reserved_", ctypes.c_int32)]


class dc_request(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int32), ("n_tris", ctypes.c_int32), ("n_pins", ctypes.c_int32),
                ("n_steps", ctypes.c_int32), ("rest_pos", ctypes.c_void_p), ("tris", ctypes.c_void_p),
                ("pins", ctypes.c_void_p), ("x0", ctypes.c_void_p), ("v0", ctypes.c_void_p),
                ("dL_dx_final", ctypes.c_void_p), ("dL_dv_final", ctypes.c_void_p), ("params", dc_params)]


class dc_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("slot", ctypes.c_int32), ("x_final", ctypes.c_void_p),
                ("v_final", ctypes.c_void_p), ("dL_dx0", ctypes.c_void_p), ("dL_dv0", ctypes.c_void_p),
                ("dL_dparams", ctypes.c_double * 3), ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_done", ctypes.c_double), ("device_bytes", ctypes.c_int64), ("device_bytes_peak", ctypes.c_int64),
                ("adj_iters", ctypes.c_int64), ("message", ctypes.c_char * 256)]


class dc_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("in_flight", ctypes.c_int64), ("peak_in_flight", ctypes.c_int64),
                ("bytes_reserved", ctypes.c_int64), ("peak_bytes_reserved", ctypes.c_int64),
                ("cloth_steps", ctypes.c_int64), ("batch_retries", ctypes.c_int64)]


KT_CLASSES = {"none": 0, "solve_fwd": 1, "solve_bwd": 2, "local": 3, "gather": 4, "front": 5, "msolve": 6,
              "krylov": 7, "apply_h": 8, "assemble": 9, "sweeps": 10}


_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
# name -> (restype, argtypes); every pointer argument is passed as a raw address
SIGNATURES = {
    "dc_create_mesh": (ctypes.c_int32, [ctypes.POINTER(_P), ctypes.c_int32, _P, ctypes.c_int32, _P,
                                        ctypes.c_int32, _P, _P]),
    "dc_create_batch": (ctypes.c_int32, [ctypes.POINTER(_P), ctypes.c_int32, _P, _P]),
    "dc_get_layout": (ctypes.c_int32, [_P, ctypes.POINTER(ctypes.c_int32), _P]),
    "dc_set_params": (ctypes.c_int32, [_P, ctypes.POINTER(dc_params)]),
    "dc_set_params_batch": (ctypes.c_int32, [_P, ctypes.c_int32, _P]),
    "dc_set_graphs": (ctypes.c_int32, [_P, ctypes.c_int32]),
    "dc_set_layout": (ctypes.c_int32, [_P, ctypes.c_int32]),
    "dc_set_instance_steps": (ctypes.c_int32, [_P, _P]),
    "dc_add_obstacle_mesh": (ctypes.c_int32, [_P, ctypes.c_int32, _P, ctypes.c_int32, _P,
                                              ctypes.POINTER(ctypes.c_int32)]),
    "dc_batch_hbm_bytes": (ctypes.c_int32, [ctypes.c_int32, _P, _P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64)]),
    "dc_autotune": (ctypes.c_int32, [_P]),
    "dc_step": (ctypes.c_int32, [_P, _P, _P, _P, _P]),
    "dc_rollout": (ctypes.c_int32, [_P, ctypes.c_int32, _P, _P, _P, _P, _P]),
    "dc_backward": (ctypes.c_int32, [_P, _P, _P, _P, _P, _P, _P]),
    "dc_global_solve": (ctypes.c_int32, [_P, _P, _P]),
    "dc_global_solve_static": (ctypes.c_int32, [_P, _P, _P]),
    "dc_debug_sweep_wait_timeout": (ctypes.c_int32, [_P, ctypes.c_int32]),
    "dc_get_instance_nonconverged": (ctypes.c_int32, [_P, _P]),
    "dc_debug_front_factor": (ctypes.c_int32, [ctypes.c_int32, ctypes.c_int32, _P, _P, _P, ctypes.c_int32,
                                               ctypes.c_int32, ctypes.c_int32]),
    "dc_get_stats": (ctypes.c_int32, [_P, ctypes.POINTER(dc_stats)]),
    "dc_fma_peak": (ctypes.c_int32, [ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]),
    "dc_set_kernel_timer": (ctypes.c_int32, [_P, ctypes.c_int32]),
    "dc_sync": (ctypes.c_int32, [_P]),
    "dc_destroy": (None, [_P]),
    "dc_last_error": (ctypes.c_char_p, [_P]),
    "dc_default_params": (None, [ctypes.POINTER(dc_params)]),
    "dc_server_create": (ctypes.c_int32, [ctypes.POINTER(_P), ctypes.POINTER(dc_server_config)]),
    "dc_server_submit": (ctypes.c_int32, [_P, ctypes.POINTER(dc_request), ctypes.POINTER(ctypes.c_int64)]),
    "dc_server_wait": (ctypes.c_int32, [_P, ctypes.c_int64, ctypes.POINTER(dc_result)]),
    "dc_server_get_stats": (ctypes.c_int32, [_P, ctypes.POINTER(dc_server_stats)]),
    "dc_server_destroy": (None, [_P]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libdc.so; raises if it has not been built (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libdc.so not found at {path}; build it with paper_2106_05306_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class DCError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def check(status, ctx=None):
    if status != DC_OK:
        msg = load().dc_last_error(ctx)
        raise DCError(status, msg.decode() if msg else "")
