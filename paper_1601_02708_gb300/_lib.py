"""ctypes declarations of the C ABI in include/lbm_ade.h (marshalling only)."""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

LBM_OK = 0
LBM_WARN_BC_INFEASIBLE = 1
LBM_ERR_NEWTON = -3
STATUS_NAMES = {0: "LBM_OK", 1: "LBM_WARN_BC_INFEASIBLE", -1: "LBM_ERR_ARG",
                -2: "LBM_ERR_CUDA", -3: "LBM_ERR_NEWTON", -4: "LBM_ERR_TIMEOUT",
                -5: "LBM_ERR_STATE", -6: "LBM_ERR_NOMEM"}


class LBMError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("precision", ctypes.c_int), ("edge", ctypes.c_int * 4),
                ("tau", ctypes.c_double), ("react_mode", ctypes.c_int),
                ("k_scalar", ctypes.c_double), ("dissolution", ctypes.c_int)]


class FemParams(ctypes.Structure):
    _fields_ = [("nex", ctypes.c_int), ("ney", ctypes.c_int),
                ("x0", ctypes.c_double), ("y0", ctypes.c_double),
                ("hx", ctypes.c_double), ("hy", ctypes.c_double),
                ("D", ctypes.c_double), ("vx", ctypes.c_double), ("vy", ctypes.c_double),
                ("theta", ctypes.c_double), ("dt", ctypes.c_double),
                ("supg", ctypes.c_int), ("tol", ctypes.c_double), ("max_iter", ctypes.c_int)]


class Diag(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("outlet_J", ctypes.c_double),
                ("outlet_flux", ctypes.c_double), ("min_f", ctypes.c_double),
                ("steps", ctypes.c_longlong), ("bc_infeasible", ctypes.c_longlong),
                ("newton_fail", ctypes.c_longlong), ("flips", ctypes.c_longlong),
                ("n_solid", ctypes.c_longlong)]


def lib_path() -> str:
    """liblbmade.so, or its debug-bounds build when LBM_ADE_DEBUG_BOUNDS=1."""
    if os.environ.get("LBM_ADE_DEBUG_BOUNDS") == "1":
        return _build.DEBUG_LIB
    return _build.LIB


def load():
    """Load liblbmade.so; raises if it has not been built (there is no
    fallback: the CUDA library is the only implementation)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(
                f"{path} is missing: build it with paper_1601_02708_gb300.build.build() "
                "(or __graft_entry__.build())")
        lib = ctypes.CDLL(path)
        P, I, D, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
        sig = {
            "lbm_init": [ctypes.POINTER(P), ctypes.POINTER(Params), P, P, P, P, P, P],
            "lbm_substeps": [P, I, I, P, P, P],
            "lbm_interface_trace": [P, I, P, P],
            "lbm_get_concentration": [P, P, I],
            "lbm_get_populations": [P, P],
            "lbm_get_solid": [P, P],
            "lbm_get_mineral": [P, P],
            "lbm_get_flip_steps": [P, P],
            "lbm_diagnostics": [P, ctypes.POINTER(Diag)],
            "lbm_set_wall_mode": [P, I],
            "lbm_min_population": [P, ctypes.POINTER(D)],
            "lbm_species_from_invariants": [ctypes.c_longlong, D, D, D, P, P, P, P, P, P],
            "lbm_invariants_from_species": [ctypes.c_longlong, D, D, D, P, P, P, P, P, P],
            "lbm_calcite_species": [ctypes.c_longlong, D, P, P, P, P, P, P],
            "lbm_calcite_invariants": [ctypes.c_longlong, P, P, P, P, P, P],
            "lbm_state_bytes": [P, ctypes.POINTER(S)],
            "lbm_save": [P, P, S],
            "lbm_restore": [P, P, S],
            "lbm_set_stream": [P, P],
            "lbm_synchronize": [P],
            "lbm_kernel_timing": [P, I],
            "lbm_set_kernel": [P, I],
            "lbm_get_kernel": [P, ctypes.POINTER(I)],
            "lbm_set_rate_field": [P, P],
            "lbm_fem_init": [ctypes.POINTER(P), ctypes.POINTER(FemParams), P, I, P, P, P],
            "lbm_fem_step": [P, P],
            "lbm_fem_interpolate": [P, I, P, P],
            "lbm_fem_get": [P, P],
            "lbm_fem_set": [P, P],
            "lbm_fem_solver_info": [P, ctypes.POINTER(I), ctypes.POINTER(D)],
            "lbm_adjoint": [P, I, I, I, P, P, P, ctypes.POINTER(D), P, P, P, P, P],
            "lbm_kernel_times_read": [P, ctypes.POINTER(D), ctypes.POINTER(ctypes.c_longlong),
                                      ctypes.POINTER(D), ctypes.POINTER(ctypes.c_longlong)],
            "lbm_init_slab": [ctypes.POINTER(P), ctypes.POINTER(Params), I, I, P, P, P, P, P, P],
            "lbm_halo_bytes": [P, I, ctypes.POINTER(S)],
            "lbm_halo_pack": [P, I, I, P],
            "lbm_halo_unpack": [P, I, I, P],
            "lbm_stage_edges": [P, P, P, P],
            "lbm_step_stream": [P, I, I, I],
            "lbm_step_dissolve": [P],
            "lbm_pair_create": [ctypes.POINTER(P), P, P],
            "lbm_pair_substeps": [P, I, I, P, P, P, P, P, P],
            "lbm1d_init": [ctypes.POINTER(P), I, D, D, I, I, P, P],
            "lbm1d_substeps": [P, I, I, P, P, P],
            "lbm1d_get": [P, P],
            "lbm1d_state_bytes": [P, ctypes.POINTER(S)],
            "lbm1d_save": [P, P, S],
            "lbm1d_restore": [P, P, S],
        }
        for name, args in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = I
        PP = ctypes.POINTER(P)
        for name, args in {
            "lbm_batch_create": [ctypes.POINTER(P), I, PP],
            "lbm_batch_substeps": [P, I, I, PP, PP, PP],
            "lbm_batch_set_shape": [P, I],
            "lbm_batch_shape_info": [I] + [ctypes.POINTER(I)] * 4,
            "lbm_batch_get_shape": [P, ctypes.POINTER(I)],
            "lbm_batch_time_steps": [P, I, ctypes.POINTER(ctypes.c_float)],
        }.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = I
        lib.lbm_batch_destroy.argtypes = [P]
        lib.lbm_batch_destroy.restype = None
        lib.lbm_batch_last_error.argtypes = []
        lib.lbm_batch_last_error.restype = ctypes.c_char_p
        lib.lbm_fem_destroy.argtypes = [P]
        lib.lbm_fem_destroy.restype = None
        lib.lbm_destroy.argtypes = [P]
        lib.lbm_destroy.restype = None
        lib.lbm_pair_destroy.argtypes = [P]
        lib.lbm_pair_destroy.restype = None
        lib.lbm1d_destroy.argtypes = [P]
        lib.lbm1d_destroy.restype = None
        lib.lbm_last_error.argtypes = []
        lib.lbm_last_error.restype = ctypes.c_char_p
        lib.lbm_abi_version.argtypes = []
        lib.lbm_abi_version.restype = I
        _lib = lib
        return lib


# The last LBM_WARN_BC_INFEASIBLE message (the library's calls that wait for
# the stream report, once per new count, boundary solves whose data had no
# non-negative solution; they are counted, not failures).
last_warning = None


def check(status: int) -> int:
    """Raise LBMError on a negative status; a warning (positive status) is
    kept in ``last_warning`` and returned."""
    global last_warning
    if status < 0:
        msg = load().lbm_last_error().decode(errors="replace")
        raise LBMError(status, msg)
    if status > 0:
        last_warning = load().lbm_last_error().decode(errors="replace")
    return status


def check_batch(status: int):
    if status != LBM_OK:
        msg = load().lbm_batch_last_error().decode(errors="replace")
        raise LBMError(status, msg)
