"""ctypes declarations of the libffadmm C ABI (include/ffadmm.h).

Argument marshalling only: every computation happens in the library.  Loading
fails loudly when the shared library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libffadmm.so")

FFA_OK = 0
STATUS_NAMES = {
    0: "FFA_OK", 1: "FFA_ERR_INVALID_ARG", 2: "FFA_ERR_DEGENERATE_ELEMENT",
    3: "FFA_ERR_SINGULAR_SYSTEM", 4: "FFA_ERR_CUDA", 5: "FFA_ERR_OOM", 6: "FFA_ERR_NAN",
    7: "FFA_ERR_NOT_INITIALIZED", 8: "FFA_ERR_FLIPPED", 9: "FFA_ERR_TIMEOUT",
}

EXPORTED = [
    "ffa_default_params", "ffa_create", "ffa_destroy", "ffa_last_error", "ffa_set_handles", "ffa_set_constraints",
    "ffa_init", "ffa_iterate", "ffa_get_W", "ffa_get_state", "ffa_set_state", "ffa_get_penalties", "ffa_energy", "ffa_gradient",
    "ffa_get_info", "ffa_last_wstep_residual", "ffa_profile_phases", "ffa_energy_noalloc",
    "ffa_forward_unrolled", "ffa_backward_unrolled",
    "ffa_batch_create", "ffa_batch_destroy", "ffa_batch_last_error", "ffa_batch_init", "ffa_batch_iterate",
    "ffa_batch_get_W", "ffa_autotune", "ffa_batch_autotune", "ffa_batch_groups", "ffa_tutte",
    "ffa_set_wait_limit", "ffa_copy_factor",
]


class Mesh(C.Structure):
    _fields_ = [("n", C.c_int32), ("m", C.c_int32), ("d", C.c_int32), ("d_in", C.c_int32),
                ("V", C.c_void_p), ("T", C.c_void_p)]


class Params(C.Structure):
    _fields_ = [("energy", C.c_int), ("rho", C.c_double), ("eps_abs", C.c_double),
                ("eps_rel", C.c_double), ("check_every", C.c_int32),
                ("require_flip_free", C.c_int32), ("local_precision", C.c_int),
                ("refine_sweeps", C.c_int32), ("nd_leaf_size", C.c_int32),
                ("host_threads", C.c_int32), ("solve_schedule", C.c_int32),
                ("penalty_schedule", C.c_int32), ("rescale_rho", C.c_double),
                ("local_variant", C.c_int32), ("solve_subtree_height", C.c_int32 * 2),
                ("prox_h", C.c_int32), ("factor_device", C.c_int32), ("top_inverse_levels", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("iters", C.c_int32), ("converged", C.c_int32), ("n_flipped", C.c_int32),
                ("checked_iter", C.c_int32), ("e_prim", C.c_double), ("e_dual", C.c_double),
                ("thr_prim", C.c_double), ("thr_dual", C.c_double), ("energy_P", C.c_double),
                ("norm_GW", C.c_double), ("norm_P", C.c_double), ("norm_GtLambda", C.c_double),
                ("rescales", C.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class Info(C.Structure):
    _fields_ = [("n", C.c_int32), ("m", C.c_int32), ("d", C.c_int32), ("d_in", C.c_int32),
                ("n_pin", C.c_int32), ("n_free", C.c_int32), ("factor_entries", C.c_int64),
                ("factor_flops", C.c_int64), ("n_supernodes", C.c_int32), ("n_levels", C.c_int32),
                ("setup_seconds_analyze", C.c_double), ("setup_seconds_factor", C.c_double),
                ("device_bytes", C.c_int64), ("bytes_local_step", C.c_int64),
                ("bytes_global_sweep", C.c_int64), ("bytes_solve_pass", C.c_int64),
                ("kernels_per_iteration", C.c_int32),
                ("kernels_per_check", C.c_int32), ("seconds_refactor", C.c_double),
                ("top_inverse_levels", C.c_int32), ("top_inverse_cols", C.c_int32),
                ("bytes_top_product", C.c_int64), ("setup_seconds_top_inverse", C.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class Tuning(C.Structure):
    _fields_ = [("local_block", C.c_int32), ("narrow_cols", C.c_int32), ("schedule", C.c_int32),
                ("bottom_levels", C.c_int32), ("ms_local", C.c_double * 3), ("ms_solve", C.c_double * 2),
                ("ms_schedule", C.c_double * 3), ("ms_bottom", C.c_double * 4),
                ("subtree_height", C.c_int32 * 2), ("ms_subtree", (C.c_double * 4) * 2)]

    def as_dict(self) -> dict:
        return {"local_block": self.local_block, "narrow_cols": self.narrow_cols, "schedule": self.schedule,
                "bottom_levels": self.bottom_levels, "ms_local": list(self.ms_local),
                "ms_solve": list(self.ms_solve), "ms_schedule": list(self.ms_schedule),
                "ms_bottom": list(self.ms_bottom), "subtree_height": list(self.subtree_height),
                "ms_subtree": [list(r) for r in self.ms_subtree]}


class PhaseTimes(C.Structure):
    _fields_ = [("reps", C.c_int32), ("ms_gather", C.c_double), ("ms_wstep", C.c_double),
                ("ms_vertex", C.c_double), ("ms_local", C.c_double), ("ms_check", C.c_double),
                ("ms_iteration", C.c_double), ("ms_solve_forward", C.c_double),
                ("ms_solve_backward", C.c_double), ("ms_top_product", C.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load() -> C.CDLL:
    """Load libffadmm.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libffadmm.so is not built ({LIB_PATH}); run "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(LIB_PATH)
    vp, i32, dbl = C.c_void_p, C.c_int32, C.c_double
    sig = {
        "ffa_default_params": ([C.POINTER(Params)], C.c_int),
        "ffa_create": ([C.POINTER(Mesh), vp, i32, vp, C.POINTER(Params), vp, C.POINTER(vp)], C.c_int),
        "ffa_destroy": ([vp], None),
        "ffa_last_error": ([vp], C.c_char_p),
        "ffa_set_handles": ([vp, vp], C.c_int),
        "ffa_set_constraints": ([vp, i32, vp, vp, vp, vp], C.c_int),
        "ffa_init": ([vp, vp], C.c_int),
        "ffa_iterate": ([vp, i32, i32, C.POINTER(Stats)], C.c_int),
        "ffa_get_W": ([vp, vp], C.c_int),
        "ffa_get_state": ([vp, vp, vp, vp], C.c_int),
        "ffa_set_state": ([vp, vp, vp, vp, vp], C.c_int),
        "ffa_get_penalties": ([vp, vp], C.c_int),
        "ffa_energy": ([vp, vp, C.POINTER(dbl)], C.c_int),
        "ffa_gradient": ([vp, vp, vp], C.c_int),
        "ffa_get_info": ([vp, C.POINTER(Info)], C.c_int),
        "ffa_copy_factor": ([vp, vp, C.c_int64], C.c_int),
        "ffa_last_wstep_residual": ([vp, C.POINTER(dbl)], C.c_int),
        "ffa_profile_phases": ([vp, i32, C.POINTER(PhaseTimes)], C.c_int),
        "ffa_energy_noalloc": ([i32, i32, i32, i32, vp, vp, vp, C.c_int, vp, vp], C.c_int),
        "ffa_forward_unrolled": ([vp, i32, i32], C.c_int),
        "ffa_backward_unrolled": ([vp, vp, vp], C.c_int),
        "ffa_batch_create": ([i32, C.POINTER(Mesh), C.POINTER(vp), vp, C.POINTER(vp), vp, vp, C.POINTER(Params), vp,
                              C.POINTER(vp)], C.c_int),
        "ffa_batch_destroy": ([vp], None),
        "ffa_batch_last_error": ([vp], C.c_char_p),
        "ffa_batch_init": ([vp, C.POINTER(vp)], C.c_int),
        "ffa_batch_iterate": ([vp, i32, i32, C.POINTER(Stats), C.POINTER(i32)], C.c_int),
        "ffa_batch_get_W": ([vp, i32, vp], C.c_int),
        "ffa_autotune": ([vp, i32, C.POINTER(Tuning)], C.c_int),
        "ffa_batch_autotune": ([vp, i32, C.POINTER(Tuning)], C.c_int),
        "ffa_batch_groups": ([vp], C.c_int32),
        "ffa_tutte": ([C.POINTER(Mesh), vp, i32, vp, C.POINTER(Params), vp, vp, C.POINTER(dbl)], C.c_int),
        "ffa_set_wait_limit": ([vp, C.c_int64], C.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


class FFAError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def check(lib: C.CDLL, ctx, status: int) -> None:
    if status != FFA_OK:
        msg = lib.ffa_last_error(ctx)
        raise FFAError(status, msg.decode() if msg else "")
