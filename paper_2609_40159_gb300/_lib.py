"""ctypes binding of the C ABI in include/sptrsv.h -- argument marshalling only.

Every function of the header is exposed under its C name.  The library is
the in-tree ``libsptrsv_gb300.so``; importing this module fails loudly if it
has not been built (there is no CPU fallback).
"""
from __future__ import annotations

import atexit
import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsptrsv_gb300.so")
# bounds-checked debug variant (built alongside; see sptrsv_checked_build)
LIB_CHECKED_PATH = os.path.join(_HERE, "libsptrsv_gb300_checked.so")

# status codes
SPTRSV_OK = 0
SPTRSV_EINVAL = 1
SPTRSV_ENOTLOWER = 2
SPTRSV_EDIAG = 3
SPTRSV_EUNSORTED = 4
SPTRSV_ETARGET = 5
SPTRSV_ENOMEM = 6
SPTRSV_ETIMEOUT = 7
SPTRSV_ECUDA = 8
SPTRSV_ENOTSUP = 9
SPTRSV_ERANGE = 10

SPTRSV_F64 = 0
SPTRSV_F32 = 1

SPTRSV_MODE_AUTO = 0
SPTRSV_MODE_LEVEL_LAUNCH = 1
SPTRSV_MODE_LEVEL_PERSISTENT = 2
SPTRSV_MODE_SYNCFREE = 3
SPTRSV_MODE_BLOCK = 4
SPTRSV_MODE_HYBRID = 5

MODE_NAMES = {
    "auto": SPTRSV_MODE_AUTO,
    "level_launch": SPTRSV_MODE_LEVEL_LAUNCH,
    "level": SPTRSV_MODE_LEVEL_PERSISTENT,
    "level_persistent": SPTRSV_MODE_LEVEL_PERSISTENT,
    "syncfree": SPTRSV_MODE_SYNCFREE,
    "block": SPTRSV_MODE_BLOCK,
    "hybrid": SPTRSV_MODE_HYBRID,
}


class sptrsv_csr(C.Structure):
    _fields_ = [
        ("n", C.c_int32),
        ("nnz", C.c_int64),
        ("row_ptr", C.c_void_p),
        ("col_idx", C.c_void_p),
        ("vals", C.c_void_p),
        ("dtype", C.c_int),
    ]


class sptrsv_csr_out(C.Structure):
    _fields_ = [("row_ptr", C.c_void_p), ("col_idx", C.c_void_p), ("vals", C.c_void_p)]


class sptrsv_plan_opts(C.Structure):
    _fields_ = [
        ("mode", C.c_int32),
        ("rows_per_warp", C.c_int32),
        ("rhs_tile", C.c_int32),
        ("build_transpose", C.c_int32),
        ("wait_limit_us", C.c_int64),
    ]


sptrsv_handle = C.c_void_p
sptrsv_plan = C.c_void_p

_P = C.c_void_p
_I32 = C.c_int32
_I64 = C.c_int64
_PI32 = C.POINTER(C.c_int32)
_PI64 = C.POINTER(C.c_int64)

# name -> (argtypes)
_SIGS = {
    "sptrsv_create": [C.POINTER(sptrsv_handle), _P],
    "sptrsv_destroy": [sptrsv_handle],
    "sptrsv_set_stream": [sptrsv_handle, _P],
    "sptrsv_get_status": [sptrsv_handle],
    "sptrsv_validate": [sptrsv_handle, C.POINTER(sptrsv_csr), _PI32],
    "sptrsv_analyze": [sptrsv_handle, C.POINTER(sptrsv_csr), _P, _P, _P, _P, _PI32,
                       C.POINTER(C.c_double)],
    "sptrsv_transpose": [sptrsv_handle, C.POINTER(sptrsv_csr), C.POINTER(sptrsv_csr_out)],
    "sptrsv_level_summary": [sptrsv_handle, C.POINTER(sptrsv_csr), _P, _P, _P, _I32, C.c_double, _P, _P, _PI64],
    "sptrsv_analyze_incremental": [sptrsv_handle, C.POINTER(sptrsv_csr), _I32, _P, _P, _P, _P, _PI32,
                                   C.POINTER(C.c_double)],
    "sptrsv_rewrite": [sptrsv_handle, C.POINTER(sptrsv_csr), _P, _P, _P, _I32, _PI64, _PI64,
                       C.POINTER(sptrsv_csr_out), C.POINTER(sptrsv_csr_out)],
    "sptrsv_plan_create": [sptrsv_handle, C.POINTER(sptrsv_csr), C.POINTER(sptrsv_csr),
                           C.POINTER(sptrsv_plan_opts), C.POINTER(sptrsv_plan)],
    "sptrsv_plan_destroy": [sptrsv_plan],
    "sptrsv_plan_info": [sptrsv_plan, _PI32, _PI32, _PI32, _PI32],
    "sptrsv_plan_set": [sptrsv_plan, _I32, _I32, _I32],
    "sptrsv_plan_set_thin_rows": [sptrsv_plan, _I32],
    "sptrsv_plan_set_blocks_per_sm": [sptrsv_plan, _I32],
    "sptrsv_solve": [sptrsv_plan, _P, _P, _I32, _I64],
    "sptrsv_solve_transpose": [sptrsv_plan, _P, _P, _I32, _I64],
    "sptrsv_solve_layout": [sptrsv_plan, _P, _P, _I32, _I64, _I32, _I32],
    "sptrsv_grad_vals": [sptrsv_plan, _P, _P, _I32, _I64, _P],
    "sptrsv_tt_apply": [sptrsv_plan, _P, _P, _I32, _I64],
    "sptrsv_batch_plan_create": [sptrsv_handle, _I32, C.POINTER(sptrsv_csr), C.POINTER(sptrsv_csr),
                                 _PI32, C.POINTER(sptrsv_plan_opts), C.POINTER(sptrsv_plan)],
    "sptrsv_batch_offsets": [sptrsv_plan, _PI64, _PI64],
    "sptrsv_batch_plan_set": [sptrsv_plan, _PI32, _PI32],
    "sptrsv_batch_plan_set_direction": [sptrsv_plan, _I32, _PI32, _PI32],
    "sptrsv_batch_plan_set_schedule": [sptrsv_plan, _I32, _PI32],
    "sptrsv_batch_solve": [sptrsv_plan, _P, _P],
    "sptrsv_batch_solve_transpose": [sptrsv_plan, _P, _P],
    "sptrsv_batch_grad_vals": [sptrsv_plan, _P, _P, _P],
    "sptrsv_batch_tt_apply": [sptrsv_plan, _P, _P],
    "sptrsv_batch_step_host": [sptrsv_plan, _P, _P, _P, _P, _P],
    "sptrsv_batch_step_wait": [sptrsv_plan],
    "sptrsv_debug_withhold_row": [sptrsv_plan, _I32],
    "sptrsv_debug_withhold_level": [sptrsv_handle, _I32, _I64],
    "sptrsv_batch_trace": [sptrsv_plan, _PI64],
    "sptrsv_solve_noalloc": [C.POINTER(sptrsv_csr), _P, _P, _I32, _I64, _P],
    "sptrsv_debug_check_index": [sptrsv_handle, _I32, _I32],
}
SPTRSV_NOALLOC_MAX_ROWS = 1 << 20
SPTRSV_BATCH_INORDER = 1
SPTRSV_ROW_MAJOR = 0
SPTRSV_COL_MAJOR = 1
SPTRSV_BATCH_LEVEL = 2

DECLARED = sorted(list(_SIGS) + ["sptrsv_status_string", "sptrsv_checked_build"])


def load(path: str = LIB_PATH):
    """Load the library and declare every signature.  Raises OSError with a
    clear message when the in-tree build is missing."""
    if not os.path.exists(path):
        raise OSError(
            f"CUDA library not built: {path} is missing (run __graft_entry__.build() or "
            "python paper_2609_40159_gb300/build.py); there is no CPU fallback")
    lib = C.CDLL(path)
    for name, args in _SIGS.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_int
    lib.sptrsv_status_string.argtypes = [C.c_int]
    lib.sptrsv_status_string.restype = C.c_char_p
    lib.sptrsv_checked_build.argtypes = []
    lib.sptrsv_checked_build.restype = C.c_int32
    return lib


_lib = None
_exiting = False


def _mark_exit():
    global _exiting
    _exiting = True


# Objects still alive when the interpreter exits (e.g. held by a traceback)
# must not call into the library from their finalisers: the CUDA runtime may
# already be torn down, and the process returns the device memory anyway.
atexit.register(_mark_exit)


def exiting() -> bool:
    return _exiting


def lib():
    global _lib
    if _lib is None:
        _lib = load()
    return _lib


class SpTRSVError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        msg = lib().sptrsv_status_string(status).decode()
        super().__init__(f"{what}: status {status} ({msg})" if what else f"status {status} ({msg})")
        self.status = status


def check(status: int, what: str = ""):
    if status != SPTRSV_OK:
        raise SpTRSVError(status, what)


def _fwd(name):
    def f(*args):
        return getattr(lib(), name)(*args)
    f.__name__ = name
    f.__doc__ = f"Direct call of the C entry point {name} (see include/sptrsv.h)."
    return f


# module-level functions with the C names
for _n in DECLARED:
    globals()[_n] = _fwd(_n)
