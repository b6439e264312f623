"""ctypes binding of libptycho (argument marshalling only).

Every function here forwards to the C ABI declared in ``include/ptycho.h``;
no step of the computation runs in Python.  Loading fails loudly when the
shared library has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libptycho.so")

PTX_OK = 0
STATUS_NAMES = {
    0: "PTX_OK",
    1: "PTX_ERR_INVALID_ARG",
    2: "PTX_ERR_UNSUPPORTED",
    3: "PTX_ERR_OUT_OF_BOUNDS",
    4: "PTX_ERR_CUDA",
    5: "PTX_ERR_TIMEOUT",
    6: "PTX_ERR_NOT_READY",
}

PTX_UPDATE_OBJ = 0x1
PTX_UPDATE_PROBE = 0x2
PTX_DM_INIT_PSI = 0x4
PTX_NO_NORMALISE = 0x8
PTX_NO_GRAPH = 0x10
PTX_ML_RESTART = 0x20
PTX_UPDATE_BACKGROUND = 0x40
PTX_FORM_TF32X2 = 0x1000
PTX_FORM_BF16X3 = 0x2000
PTX_FORM_BF16X2 = 0x4000
PTX_MAX_MODES = 8
PTX_ALGO_AP = 0
PTX_ALGO_DM = 1
SUPPORTED_SIZES = (8, 12, 16, 32, 64, 80, 128, 160, 192, 224, 256, 384, 400, 448, 512)

# Every symbol include/ptycho.h declares.
EXPORTS = (
    "ptx_workspace_bytes", "ptx_create", "ptx_ap_cycles", "ptx_dm_cycles", "ptx_cycles", "ptx_llk", "ptx_ml_grad",
    "ptx_ml_cycles", "ptx_ml_line_coeffs", "ptx_position_shifts", "ptx_set_positions",
    "ptx_normalise", "ptx_accumulators", "ptx_set_param", "ptx_fft2", "ptx_profile_enable", "ptx_profile_read",
    "ptx_llk_static", "ptx_counts_to_float", "ptx_encode_counts8", "ptx_counts8_to_float", "ptx_wait_selftest",
    "ptx_fma_peak", "ptx_accumulate_shifts", "ptx_cycle_kernels",
    "ptx_last_error", "ptx_destroy",
)
KERNEL_KINDS = ("row_fwd", "col", "row_bwd", "den_max", "normalise", "cycle_end", "obj_gather")
PTX_STAGE_PROBE = 0x100
PTX_STAGE_OBJ_GATHER = 0x200
PTX_STAGE_OBJ_NORMALISE = 0x400


class PtychoError(RuntimeError):
    """A libptycho call returned an error status."""

    def __init__(self, status: int, message: str):
        self.status = status
        self.status_name = STATUS_NAMES.get(status, str(status))
        super().__init__(f"{self.status_name}: {message}")


class Problem(ctypes.Structure):
    """Mirror of ``ptx_problem``."""

    _fields_ = [
        ("N", ctypes.c_int32),
        ("K", ctypes.c_int32),
        ("J", ctypes.c_int32),
        ("Ho", ctypes.c_int32),
        ("Wo", ctypes.c_int32),
        ("obj", ctypes.c_void_p),
        ("probe", ctypes.c_void_p),
        ("positions", ctypes.c_void_p),
        ("iobs", ctypes.c_void_p),
        ("mask", ctypes.c_void_p),
        ("psi", ctypes.c_void_p),
        ("nearfield", ctypes.c_double),
        ("background", ctypes.c_void_p),
    ]


_lib = None


def load(path: str | None = None):
    """Load libptycho.so (once).  Raises if it is missing: build it first with
    ``python -c 'import __graft_entry__ as g; g.build()'`` or
    ``python paper_2008_11511_gb300/build.py``."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libptycho.so not found at {p}: build it with paper_2008_11511_gb300/build.py")
    lib = ctypes.CDLL(p)
    vp, i32, u32, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32, ctypes.c_size_t
    st = ctypes.c_int
    sig = {
        "ptx_workspace_bytes": (st, [ctypes.POINTER(Problem), i32, ctypes.POINTER(sz)]),
        "ptx_create": (st, [ctypes.POINTER(vp), ctypes.POINTER(Problem), i32, vp, sz, vp]),
        "ptx_ap_cycles": (st, [vp, i32, u32, vp, vp]),
        "ptx_dm_cycles": (st, [vp, i32, u32, vp, vp]),
        "ptx_cycles": (st, [vp, i32, u32, vp, vp, vp]),
        "ptx_llk": (st, [vp, vp, vp]),
        "ptx_ml_grad": (st, [vp, vp, vp, vp, vp]),
        "ptx_ml_cycles": (st, [vp, i32, u32, vp, vp]),
        "ptx_ml_line_coeffs": (st, [vp, vp, vp, vp, vp]),
        "ptx_normalise": (st, [vp, u32, vp]),
        "ptx_accumulators": (st, [vp, i32, ctypes.POINTER(vp), ctypes.POINTER(sz), ctypes.POINTER(vp),
                                  ctypes.POINTER(sz)]),
        "ptx_set_param": (st, [vp, ctypes.c_char_p, ctypes.c_double]),
        "ptx_fft2": (st, [vp, i32, i32, i32, vp]),
        "ptx_profile_enable": (st, [vp, i32]),
        "ptx_profile_read": (st, [vp, i32, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)]),
        "ptx_llk_static": (st, [i32, i32, i32, i32, i32, vp, vp, vp, vp, vp, vp, vp]),
        "ptx_counts_to_float": (st, [vp, vp, sz, vp]),
        "ptx_encode_counts8": (st, [vp, sz, vp, vp, vp, sz, ctypes.POINTER(sz)]),
        "ptx_counts8_to_float": (st, [vp, vp, sz, vp, vp, sz, vp]),
        "ptx_wait_selftest": (st, [vp, i32, vp]),
        "ptx_fma_peak": (st, [i32, i32, vp, ctypes.POINTER(ctypes.c_double), vp]),
        "ptx_cycle_kernels": (st, [vp, i32, u32, ctypes.POINTER(ctypes.c_int64)]),
        "ptx_accumulate_shifts": (st, [i32, vp, ctypes.c_double, ctypes.c_double, i32, i32, vp, vp,
                                       ctypes.POINTER(i32)]),
        "ptx_last_error": (ctypes.c_char_p, []),
        "ptx_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def check(status: int):
    if status != PTX_OK:
        msg = load().ptx_last_error()
        raise PtychoError(status, msg.decode() if msg else "")


def call(name: str, *args):
    """Call ``name`` and raise PtychoError on a non-zero status."""
    check(getattr(load(), name)(*args))
