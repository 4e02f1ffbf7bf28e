"""ctypes declarations of the C ABI in include/sphmesh.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os
import re
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libsphmesh.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "sphmesh.h")

SPH_OK = 0
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "OOM", 3: "CUDA", 4: "NONFINITE", 5: "OUT_OF_DOMAIN",
                6: "CELL_OVERFLOW", 7: "TIMEOUT", 8: "STATE"}
SPH_PREC_FP32_SPLIT = 0
SPH_PREC_FP64 = 1
SPH_OUT_RHO, SPH_OUT_ACC, SPH_OUT_VISC = 0, 1, 2


class sph_shape(C.Structure):
    _fields_ = [("kind", C.c_int32), ("keep_inside", C.c_int32),
                ("center", C.c_double * 3), ("size", C.c_double * 3)]


class sph_domain(C.Structure):
    _fields_ = [("dim", C.c_int32), ("n_shapes", C.c_int32), ("lo", C.c_double * 3),
                ("hi", C.c_double * 3), ("shapes", sph_shape * 4)]


class sph_field(C.Structure):
    _fields_ = [("kind", C.c_int32), ("dist_shape", C.c_int32), ("s0", C.c_double), ("a", C.c_double),
                ("b", C.c_double), ("n_poly", C.c_int32), ("reserved", C.c_int32),
                ("poly", C.c_double * 8), ("rho_scale", C.c_double)]


class sph_params(C.Structure):
    _fields_ = [("P0", C.c_double), ("gamma", C.c_double), ("sigma0", C.c_double), ("tau", C.c_double),
                ("kappa", C.c_double), ("precision", C.c_int32), ("kernel_id", C.c_int32),
                ("seed", C.c_uint64), ("cell_factor", C.c_double), ("block_size", C.c_int32),
                ("use_graph", C.c_int32), ("record_fields", C.c_int32), ("list_capacity", C.c_int32),
                ("skin", C.c_double)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p)


class sph_alloc(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", C.c_void_p)]


class sph_stats(C.Structure):
    _fields_ = [("step", C.c_int64), ("sigma", C.c_double), ("dt1", C.c_double), ("dt2", C.c_double),
                ("min_rc_over_a", C.c_double), ("max_a", C.c_double), ("sum_rho", C.c_double),
                ("err_l2", C.c_double), ("err_max", C.c_double), ("interface_pairs", C.c_int64),
                ("force_pairs", C.c_int64), ("wall_moved", C.c_int64), ("rho_scale", C.c_double),
                ("error_flags", C.c_int32), ("n_levels", C.c_int32),
                ("list_entries", C.c_int64), ("list_rebuilds", C.c_int64), ("list_max", C.c_int32),
                ("list_capacity", C.c_int32), ("ramp_t0", C.c_double), ("ramp_t1", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class sph_background(C.Structure):
    _fields_ = [("dims", C.c_int32 * 3), ("reserved", C.c_int32), ("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("phi", C.c_void_p), ("spacing", C.c_void_p)]


class sph_grid_info(C.Structure):
    _fields_ = [("n_levels", C.c_int32), ("dim", C.c_int32), ("lo", C.c_double * 3), ("h0", C.c_double),
                ("lip_h", C.c_double), ("cell", C.c_double * 8), ("dims", (C.c_int32 * 3) * 8),
                ("base", C.c_uint32 * 9)]


class sph_objective(C.Structure):
    _fields_ = [("density_weight", C.c_double), ("lambda_", C.c_double), ("frozen_dt", C.c_int32),
                ("ckpt_every", C.c_int32)]


class sph_grad(C.Structure):
    _fields_ = [("L", C.c_double), ("d_sigma0", C.c_double), ("d_gamma", C.c_double), ("d_P0", C.c_double),
                ("d_poly", C.c_double * 8)]


class sph_batch_trial(C.Structure):
    _fields_ = [("branches", C.c_int32), ("pass_threads", C.c_int32), ("cell_factor", C.c_double),
                ("ms_per_step", C.c_float), ("stage_views", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if not k.startswith("reserved")}


class sph_instance_desc(C.Structure):
    _fields_ = [("dom", sph_domain), ("field", sph_field), ("n_particles", C.c_int64), ("n_colors", C.c_int32),
                ("reserved", C.c_int32), ("params", sph_params)]


H = C.c_void_p
_lock = threading.Lock()
_lib = None


def declared_symbols():
    """Every function name declared in include/sphmesh.h."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?(?:sph_status|void|const char\s*\*)\s*(sph_\w+)\s*\(",
                                 txt, flags=re.M)))


def load():
    """Load libsphmesh.so (built by paper_1906_07925_gb300.build). Raises if missing:
    there is no fallback implementation."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        P = C.POINTER
        sig = {
            "sph_create": [P(sph_domain), P(sph_field), C.c_int64, C.c_int32, P(sph_params), P(sph_alloc),
                           C.c_void_p, P(H)],
            "sph_set_surface": [H, C.c_void_p],
            "sph_create_background": [P(sph_domain), P(sph_field), P(sph_background), C.c_int64, C.c_int32,
                                      P(sph_params), P(sph_alloc), C.c_void_p, P(H)],
            "sph_set_state": [H, C.c_void_p, C.c_void_p, C.c_int32],
            "sph_step": [H, C.c_int32],
            "sph_step_profiled": [H, C.c_int32, P(C.c_float)],
            "sph_ramp_surface_tension": [H, C.c_int64, C.c_int64],
            "sph_auto_ramp": [H, C.c_int32, C.c_double, C.c_double],
            "sph_get_positions": [H, C.c_void_p, C.c_int32],
            "sph_get_colors": [H, C.c_void_p, C.c_int32],
            "sph_get_stats": [H, P(sph_stats)],
            "sph_get_field": [H, C.c_int32, C.c_void_p, C.c_int32],
            "sph_neighbor_sets": [H, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
            "sph_get_cell_list": [H, C.c_void_p, C.c_void_p],
            "sph_get_grid": [H, P(sph_grid_info)],
            "sph_sync": [H],
            "sph_save": [H, C.c_void_p, P(C.c_size_t)],
            "sph_load": [H, C.c_void_p, C.c_size_t],
            "sph_get_info": [H, P(C.c_int64), P(C.c_int32), P(C.c_double)],
            "sph_backward": [H, C.c_int32, P(sph_objective), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                             C.c_int32, P(sph_grad)],
            "sph_batch_create": [C.c_void_p, C.c_int32, P(sph_alloc), C.c_void_p, C.c_int32, P(H)],
            "sph_batch_tune": [H, C.c_void_p, C.c_int32, C.c_int32],
            "sph_batch_step": [H, C.c_int32],
            "sph_batch_step_each": [H, C.c_int32],
            "sph_batch_get": [H, C.c_int32, P(H)],
            "sph_batch_info": [H, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
            "sph_batch_sync": [H],
            "sph_batch_tuning": [H, P(sph_batch_trial), C.c_void_p, C.c_int32, P(C.c_int32)],
            "sph_set_tuning": [H, C.c_int32, C.c_double, C.c_int32],
            "sph_get_tuning": [H, P(C.c_int32), P(C.c_double), P(C.c_int32)],
            "sph_get_stage_info": [H, P(C.c_int64), P(C.c_int64), P(C.c_int64)],
            "sph_get_color_volumes": [H, C.c_void_p, C.c_void_p],
            "sph_eval_forces_noalloc": [P(sph_domain), P(sph_field), P(sph_params), C.c_int64, C.c_void_p,
                                        C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.sph_last_error.argtypes = [H]
        L.sph_last_error.restype = C.c_char_p
        L.sph_destroy.argtypes = [H]
        L.sph_destroy.restype = None
        L.sph_batch_destroy.argtypes = [H]
        L.sph_batch_destroy.restype = None
        L.sph_batch_last_error.argtypes = [H]
        L.sph_batch_last_error.restype = C.c_char_p
        _lib = L
        return L
