"""ctypes binding of ``libhram.so`` (the C-ABI declared in include/hram.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  Importing this module does not need a GPU; loading the library
does not either, but every compute call does.  There is no CPU fallback: if
the library is missing, :func:`lib` raises.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# HRAM_CHECKED=1 selects the bounds-checked build of the same library (every
# cell-list, sorted-array and ghost index checked before use; HR_ECHECK on a
# failure); it computes the same step
CHECKED = os.environ.get("HRAM_CHECKED", "0") == "1"
LIB_PATH = os.path.join(HERE, "libhram_checked.so" if CHECKED else "libhram.so")
MAX_PROBES = 16

# status codes (hram.h)
HR_OK = 0
HR_EINVAL = -1
HR_ENOMEM = -2
HR_ECUDA = -3
HR_ENAN = -4
HR_EDT = -5
HR_ETIMEOUT = -6
HR_ERANGE = -7
HR_EIO = -8
HR_ECHECK = -9
HR_WPENETRATION = 1
HR_WOUTSIDE = 2
HR_WPROBEFULL = 4
HR_FLAG_TIMING = 1
HR_FLAG_TANGENT = 2
HR_FLAG_STAGE_POS = 4
HR_FLAG_STAGE_ALL = 8
HR_FLAG_NEWTON3 = 16
HR_FLAG_PASS_LANES2 = 32
HR_FLAG_PASS_LANES4 = 64
HR_FLAG_PASS_SPLIT = 128
HR_FLAG_PASS_FUSED = 256
HR_FLAG_CLOSE_INLINE = 512

EXPORTS = (
    "hr_workspace_bytes", "hr_init_case", "hr_step", "hr_run", "hr_sync", "hr_probe_pressure",
    "hr_probe_times", "hr_diagnostics", "hr_diag_history", "hr_get_state", "hr_set_state",
    "hr_get_energy", "hr_get_ghosts", "hr_get_scalars", "hr_case_info", "hr_debug_neighbors",
    "hr_kernel_times", "hr_save_state", "hr_load_state", "hr_tangent_outputs",
    "hr_adjoint_forward", "hr_adjoint_backward",
    "hr_neighbor_counts_static", "hr_batch_create", "hr_batch_step", "hr_batch_run",
    "hr_batch_done", "hr_batch_destroy", "hr_batch_create_persistent", "hr_persist_capacity",
    "hr_fp32_rate", "hr_destroy", "hr_status_str",
)
HR_STATIC_NEIGHBOR_MAX = 1 << 21


class HrParams(C.Structure):
    _fields_ = [
        ("dx", C.c_double), ("h_over_dx", C.c_double), ("Lx", C.c_double), ("W", C.c_double),
        ("wall_layers", C.c_int32), ("end_walls", C.c_int32),
        ("R_disk", C.c_double), ("v0", C.c_double), ("tau", C.c_double), ("t_ramp", C.c_double),
        ("x_c0", C.c_double), ("y_c0", C.c_double),
        ("Ng", C.c_int32), ("motion", C.c_int32),
        ("a_const", C.c_double), ("drag_M", C.c_double), ("drag_Cd", C.c_double),
        ("drag_R", C.c_double),
        ("rho0", C.c_double), ("c0", C.c_double), ("gamma", C.c_double), ("p_cav", C.c_double),
        ("alpha", C.c_double), ("eta2", C.c_double), ("eps_xsph", C.c_double),
        ("mu_lam", C.c_double), ("gx", C.c_double), ("gy", C.c_double), ("cfl", C.c_double),
        ("dt_mode", C.c_int32), ("n_probes", C.c_int32),
        ("rho_lo", C.c_double), ("rho_hi", C.c_double), ("box_pad", C.c_double),
        ("cell_factor", C.c_double),
        ("probe_xy", C.c_double * (2 * MAX_PROBES)),
        ("probe_capacity", C.c_int64),
        ("diag_every", C.c_int32), ("flags", C.c_int32),
        ("disk_density", C.c_double),
        ("closure", C.c_int32),
        ("mg_S1", C.c_double), ("mg_gamma0", C.c_double), ("mg_a", C.c_double),
        ("mg_mu_max", C.c_double),
        ("wall_reflect", C.c_int32),
    ]


class HrDiag(C.Structure):
    _fields_ = [(n, C.c_double) for n in (
        "mass", "px", "py", "KE", "PE", "E_el", "rho_min", "rho_max", "p_min", "p_max",
        "vmax_fluid", "n_in", "penetrated", "t", "dt", "W_boundary", "wall_impulse",
        "dissipation", "step")]


_lib = None


def lib() -> C.CDLL:
    """The loaded library with argument types set; raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libhram.so is not built (run python -m paper_2609_05494_b300.build); "
                           "there is no CPU fallback")
    L = C.CDLL(LIB_PATH)
    vp, i64, P = C.c_void_p, C.c_int64, C.POINTER
    L.hr_workspace_bytes.argtypes = [P(HrParams), i64, P(C.c_size_t)]
    L.hr_init_case.argtypes = [P(HrParams), vp, i64, vp, vp, vp, C.c_size_t, vp, P(vp)]
    L.hr_step.argtypes = [vp]
    L.hr_run.argtypes = [vp, i64, C.c_double]
    L.hr_sync.argtypes = [vp]
    L.hr_probe_pressure.argtypes = [vp, vp, i64, P(i64)]
    L.hr_probe_times.argtypes = [vp, vp, i64, P(i64)]
    L.hr_diagnostics.argtypes = [vp, P(HrDiag)]
    L.hr_diag_history.argtypes = [vp, vp, i64, P(i64)]
    L.hr_get_state.argtypes = [vp, vp, vp, vp, vp, i64]
    L.hr_set_state.argtypes = [vp, vp, vp, vp, i64]
    L.hr_get_energy.argtypes = [vp, vp, vp, i64]
    L.hr_get_ghosts.argtypes = [vp, vp, vp, vp, vp, i64]
    L.hr_get_scalars.argtypes = [vp, vp, C.c_int]
    L.hr_case_info.argtypes = [vp, vp, C.c_int]
    L.hr_debug_neighbors.argtypes = [vp, vp, vp, i64, P(i64)]
    L.hr_kernel_times.argtypes = [vp, vp, C.c_int]
    L.hr_save_state.argtypes = [vp, C.c_char_p]
    L.hr_load_state.argtypes = [vp, C.c_char_p]
    L.hr_tangent_outputs.argtypes = [vp, vp, C.c_int]
    L.hr_adjoint_forward.argtypes = [vp, i64, C.c_int32, vp, C.c_int]
    L.hr_adjoint_backward.argtypes = [vp, vp, C.c_int]
    L.hr_neighbor_counts_static.argtypes = [vp, vp, i64]
    L.hr_batch_create.argtypes = [vp, C.c_int, C.c_double, C.c_int, vp, P(vp)]
    L.hr_batch_create_persistent.argtypes = [vp, C.c_int, C.c_double, vp, i64, vp, P(vp)]
    L.hr_persist_capacity.argtypes = [C.c_int, P(C.c_int32)]
    L.hr_fp32_rate.argtypes = [C.c_int, vp, P(C.c_double)]
    L.hr_batch_step.argtypes = [vp]
    L.hr_batch_run.argtypes = [vp, i64, P(i64)]
    L.hr_batch_done.argtypes = [vp, P(C.c_int)]
    L.hr_batch_destroy.argtypes = [vp]
    L.hr_batch_destroy.restype = None
    L.hr_destroy.argtypes = [vp]
    L.hr_destroy.restype = None
    L.hr_status_str.argtypes = [C.c_int]
    L.hr_status_str.restype = C.c_char_p
    for name in EXPORTS:
        if name not in ("hr_destroy", "hr_status_str", "hr_batch_destroy"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


class HramError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = lib().hr_status_str(code).decode()
        super().__init__("%s: %s (%d)" % (where, msg, code))
        self.code = code


def check(code: int, where: str) -> int:
    if code < 0:
        raise HramError(code, where)
    return code
