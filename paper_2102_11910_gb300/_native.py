"""ctypes loader of the gridpf C-ABI library (libgridpf.so).

There is no fallback: if the library is missing or fails to load, every call
raises.  Build it with ``paper_2102_11910_gb300.build.build()``.
"""
import ctypes
import os
import re

from . import build as _build

_LIB = None

# C signatures of the entry points declared in include/gridpf.h
_c = ctypes
_P = _c.c_void_p
_D = _c.c_double
_I64 = _c.c_int64
_I32 = _c.c_int32
SIGNATURES = {
    "pf_plan_create": (_c.c_int, [_P, _P, _c.POINTER(_P)]),
    "pf_plan_destroy": (_c.c_int, [_P]),
    "pf_plan_fft_size": (_c.c_int, [_P, _c.POINTER(_I32), _c.POINTER(_I32)]),
    "pf_lgf_table": (_c.c_int, [_P, _P]),
    "pf_sync": (_c.c_int, [_P, _c.POINTER(_I64)]),
    "pf_last_error": (_c.c_char_p, [_P]),
    "pf_timing_enable": (_c.c_int, [_P, _I32]),
    "pf_timing_report": (_c.c_int, [_P, _c.c_char_p, _I64]),
    "pf_launch_config_get": (_c.c_int, [_P, _P]),
    "pf_launch_config_set": (_c.c_int, [_P, _P]),
    "pf_autotune": (_c.c_int, [_P, _I64, _c.c_char_p, _I32, _P, _P]),
    "pf_regularize": (_c.c_int, [_P, _P, _P, _P, _I64, _P]),
    "pf_poisson_solve": (_c.c_int, [_P, _P, _P]),
    "pf_velocity_solve": (_c.c_int, [_P, _P, _D, _D, _P]),
    "pf_interpolate": (_c.c_int, [_P, _P, _P, _P, _I64, _P, _P]),
    "pf_vic_velocity": (_c.c_int, [_P, _P, _P, _P, _I64, _D, _D, _P, _P]),
    "pf_vic_velocity_host": (_c.c_int, [_P, _P, _P, _P, _I64, _D, _D, _P, _P]),
    "pf_vic_velocity_host_async": (_c.c_int, [_P, _P, _P, _P, _I64, _D, _D, _P, _P]),
    "pf_vic_state_create": (_c.c_int, [_P, _I64, _c.POINTER(_P)]),
    "pf_vic_state_destroy": (_c.c_int, [_P]),
    "pf_vic_state_set": (_c.c_int, [_P, _P, _P, _P, _I64]),
    "pf_vic_state_get": (_c.c_int, [_P, _P, _P, _P, _c.POINTER(_I64), _c.POINTER(_D)]),
    "pf_vic_step": (_c.c_int, [_P, _D, _D, _D, _P, _P]),
    "pf_regularize_noalloc": (_c.c_int, [_P, _P, _P, _P, _I64, _P, _P, _P, _P]),
    "pf_schur_factor": (_c.c_int, [_P, _P, _c.POINTER(_P)]),
    "pf_schur_destroy": (_c.c_int, [_P]),
    "pf_schur_info": (_c.c_int, [_P, _P, _P, _P]),
    "pf_sheet_solve": (_c.c_int, [_P, _P, _P, _P, _I32, _D, _I32, _P, _P, _P, _P, _P, _P]),
    "pf_sheet_solve_vortices": (_c.c_int, [_P, _P, _P, _P, _P, _I64, _P, _I32, _D, _I32, _P, _P, _P, _P, _P, _P]),
    "pf_impulse": (_c.c_int, [_P, _P, _P, _P, _P, _P, _P, _P]),
    "pf_plan_set_rhs_route": (_c.c_int, [_P, _I32]),
    "pf_sheet_solve_edges": (_c.c_int, [_P, _P, _P, _P, _D, _I32, _P, _P, _P, _P, _P, _P, _P]),
    "pf_sheet_solve_multi": (_c.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "pf_step_multi": (_c.c_int, [_P, _P, _I32, _P, _D, _I32]),
    "pf_sheet_regularize": (_c.c_int, [_P, _P, _P, _P]),
    "pf_pressure_setup": (_c.c_int, [_P, _P, _P, _P]),
    "pf_potential_jump": (_c.c_int, [_P, _P, _P, _P]),
    "pf_pressure_jump": (_c.c_int, [_P, _P, _P, _P, _P, _P, _D, _P]),
    "pf_pressure_field": (_c.c_int, [_P, _P, _P, _P, _P, _P, _P, _D, _P]),
    "pf_state_create": (_c.c_int, [_P, _I64, _c.POINTER(_P)]),
    "pf_state_destroy": (_c.c_int, [_P]),
    "pf_state_set": (_c.c_int, [_P, _P, _P, _P, _I64, _D]),
    "pf_state_get": (_c.c_int, [_P, _P, _P, _P, _c.POINTER(_I64), _c.POINTER(_D)]),
    "pf_step": (_c.c_int, [_P, _P, _P, _D, _I32]),
    "pf_step_batch": (_c.c_int, [_I32, _P, _P, _P, _P, _I32]),
    "pf_batch_create": (_c.c_int, [_I32, _P, _P, _P, _P, _I32, _P]),
    "pf_batch_step": (_c.c_int, [_P, _I32]),
    "pf_batch_destroy": (_c.c_int, [_P]),
    "pf_plan_clone": (_c.c_int, [_P, _I32, _P, _c.POINTER(_P)]),
    "pf_server_create": (_c.c_int, [_P, _c.POINTER(_P)]),
    "pf_server_destroy": (_c.c_int, [_P]),
    "pf_server_submit": (_c.c_int, [_P, _P, _c.POINTER(_I64)]),
    "pf_server_progress": (_c.c_int, [_P, _I32, _P, _c.POINTER(_I32)]),
    "pf_server_result": (_c.c_int, [_P, _I64, _P, _P, _P, _c.POINTER(_I64), _c.POINTER(_D)]),
    "pf_server_stats": (_c.c_int, [_P, _c.POINTER(_I32), _c.POINTER(_I32), _c.POINTER(_I64)]),
}

STATUS = {0: "PF_OK", 1: "PF_ERR_ARG", 2: "PF_ERR_OOM", 3: "PF_ERR_CUDA", 4: "PF_ERR_OUT_OF_DOMAIN",
          5: "PF_ERR_SINGULAR", 6: "PF_ERR_TIMEOUT", 7: "PF_ERR_NOT_FACTORED", 8: "PF_ERR_CAPACITY",
          9: "PF_ERR_INTERNAL"}


class GridPfError(RuntimeError):
    def __init__(self, status, where, detail=""):
        self.status = status
        self.name = STATUS.get(status, str(status))
        self.detail = detail
        super().__init__("%s returned %s%s" % (where, self.name, (": " + detail) if detail else ""))


class PfGridDesc(ctypes.Structure):
    _fields_ = [("nx", _I32), ("ny", _I32), ("dx", _D), ("x0", _D), ("y0", _D), ("precision", _I32)]


class PfLaunchConfig(ctypes.Structure):
    _fields_ = [("tile", _I32), ("min_span", _I32), ("tile_threads", _I32), ("fft", _I32)]


class PfBodyDesc(ctypes.Structure):
    _fields_ = [("ns", _I32), ("x", _P), ("y", _P), ("ds", _P)]


class PfMotion(ctypes.Structure):
    _fields_ = [("U", _D), ("V", _D), ("Omega", _D), ("Uinf", _D), ("Vinf", _D)]


MAX_BODIES = 4


class PfMultibody(ctypes.Structure):
    _fields_ = [("n_bodies", _I32), ("start", _I32 * (MAX_BODIES + 1)), ("n_edges", _I32 * MAX_BODIES),
                ("edge", (_I32 * 2) * MAX_BODIES), ("motion", PfMotion * MAX_BODIES), ("gamma_w", _D * MAX_BODIES)]


class PfBodyKinematics(ctypes.Structure):
    _fields_ = [("ns", _I32), ("xb", _P), ("yb", _P), ("ds", _P), ("n_edges", _I32), ("edge", _I32 * 2),
                ("alpha0", _D), ("amp", _D), ("omega", _D), ("Uinf", _D), ("Vinf", _D),
                ("edge_bounded", _I32), ("edge_bounds", _D * 4)]


class PfServerConfig(ctypes.Structure):
    _fields_ = [("max_slots", _I32), ("hbm_budget_bytes", _I64), ("precision", _I32)]


class PfRequest(ctypes.Structure):
    _fields_ = [("grid", PfGridDesc), ("body", PfBodyKinematics), ("X", _P), ("Y", _P), ("Gam", _P), ("nv", _I64),
                ("capacity", _I64), ("nsteps", _I32), ("dt", _D), ("scheme", _I32)]


def header_path():
    return os.path.join(_build.ROOT, "include", "gridpf.h")


def declared_functions():
    """Names of the functions declared in include/gridpf.h."""
    txt = open(header_path()).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(pf_[a-z0-9_]+)\s*\(", txt, flags=re.M)))


def lib():
    """Load (building first if needed) and return the ctypes library."""
    global _LIB
    if _LIB is None:
        path = _build.build()
        try:
            L = ctypes.CDLL(path)
        except OSError as e:
            raise RuntimeError("gridpf CUDA library could not be loaded from %s: %s" % (path, e))
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def check(status, where, plan=None):
    if status != 0:
        detail = ""
        if plan is not None:
            msg = lib().pf_last_error(plan)
            detail = msg.decode() if msg else ""
        raise GridPfError(status, where, detail)
