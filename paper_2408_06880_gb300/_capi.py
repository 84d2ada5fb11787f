"""ctypes declarations of the C ABI in include/sparse_lbm.h (marshalling only).

Loading fails loudly when the compiled library is missing: there is no CPU or
eager-PyTorch fallback for any step of the method."""
from __future__ import annotations

import ctypes as C
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libsparse_lbm.so")

OK, EINVAL, ENOMEM, ECUDA, EUNSUPPORTED, EDIVERGED, ETIMEOUT, EABORTED, EDEVICE = range(9)
SRT, TRT, MRT, CM, CUMULANT = 0, 1, 2, 3, 4
FP32, FP16, BF16 = 0, 1, 2
SPARSE, DENSE, SPARSE_PULL = 0, 1, 2
ORDER_LEX, ORDER_BRICK8, ORDER_HYBRID = 0, 1, 2
MEM_DEVICE, MEM_HOST = 0, 1
ORDER_CELLS, ORDER_VOXELS = 0, 1
NOALLOC_MAX_VOXELS = 268435456
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "EUNSUPPORTED", 5: "EDIVERGED",
                6: "ETIMEOUT", 7: "EABORTED", 8: "EDEVICE"}


class SlbmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Desc(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("flags", C.c_void_p),
                ("periodic", C.c_uint32), ("q", C.c_int32), ("op", C.c_int32),
                ("omega_plus", C.c_double), ("trt_magic", C.c_double), ("force", C.c_double * 3),
                ("inlet_u", C.c_void_p), ("n_inlet_u", C.c_int64), ("rho_out", C.c_double),
                ("storage", C.c_int32), ("scale_exp", C.c_int32), ("layout", C.c_int32),
                ("order", C.c_int32)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class Allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", C.c_void_p)]


class Info(C.Structure):
    _fields_ = [("n_voxels", C.c_int64), ("n_fluid", C.c_int64), ("stride", C.c_int64),
                ("n_bc_links", C.c_int64), ("device_bytes", C.c_int64), ("step", C.c_int64),
                ("q", C.c_int32), ("op", C.c_int32), ("storage", C.c_int32), ("layout", C.c_int32),
                ("scale_exp", C.c_int32), ("pad", C.c_int32)]


# name -> (restype, argtypes); every entry point declared in include/sparse_lbm.h
_vp, _i32, _i64, _st = C.c_void_p, C.c_int32, C.c_int64, C.c_int
SIGNATURES = {
    "sparse_lbm_create": (_st, [C.POINTER(Desc), C.POINTER(Allocator), _vp, C.POINTER(_vp)]),
    "sparse_lbm_step": (_st, [_vp, _i32]),
    "sparse_lbm_step_graph": (_st, [_vp, _i32]),
    "sparse_lbm_macroscopic": (_st, [_vp, _vp, _vp, _i32, _i32]),
    "sparse_lbm_reduce": (_st, [_vp, _vp, _i32]),
    "sparse_lbm_reduce_ext": (_st, [_vp, _vp, _i32]),
    "sparse_lbm_set_storage": (_st, [_vp, _i32, _i32]),
    "sparse_lbm_init_equilibrium": (_st, [_vp, _vp, _vp, _i32, _i32]),
    "sparse_lbm_info": (_st, [_vp, C.POINTER(Info)]),
    "sparse_lbm_export_lists": (_st, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "sparse_lbm_export_codes": (_st, [_vp, _vp, _vp]),
    "sparse_lbm_state_bytes": (_st, [_vp, C.POINTER(_i64)]),
    "sparse_lbm_get_state": (_st, [_vp, _vp, C.POINTER(_i64)]),
    "sparse_lbm_set_state": (_st, [_vp, _vp, _i64]),
    "sparse_lbm_set_launch": (_st, [_vp, _i32, _i32, _i32, _i32]),
    "sparse_lbm_set_mrt_rates": (_st, [_vp, _vp]),
    "sparse_lbm_set_cm_rates": (_st, [_vp, C.c_double, C.c_double]),
    "sparse_lbm_set_checked": (_st, [_vp, _i32]),
    "sparse_lbm_device_error": (_st, [_vp, C.POINTER(_i32)]),
    "sparse_lbm_free": (None, [_vp]),
    "sparse_lbm_last_error": (C.c_char_p, []),
    "sparse_lbm_compact_noalloc": (_st, [_vp, _i64, _vp, _vp, _vp, _vp]),
    "slbm_pool_create": (_st, [_i32, _i32, _i32, _vp, C.POINTER(_vp)]),
    "slbm_pool_add": (_st, [_vp, _vp, C.POINTER(_i32)]),
    "slbm_pool_remove": (_st, [_vp, _i32]),
    "slbm_pool_step": (_st, [_vp, _i32, _i32]),
    "slbm_pool_reduce": (_st, [_vp, _vp, _i32]),
    "slbm_pool_reduce_ext": (_st, [_vp, _vp, _i32]),
    "slbm_pool_set_launch": (_st, [_vp, _i32, _i32]),
    "slbm_pool_abort": (_st, [_vp, _i32]),
    "slbm_pool_set_split": (_st, [_vp, _i64]),
    "slbm_pool_set_group_bytes": (_st, [_vp, _i64]),
    "slbm_pool_set_streams": (_st, [_vp, _i32]),
    "slbm_pool_free": (None, [_vp]),
}

_lib = None


def lib():
    """Load the library (once).  Raises ImportError if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'`; "
                              "there is no fallback implementation")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(status: int) -> None:
    if status != OK:
        msg = lib().sparse_lbm_last_error() or b""
        raise SlbmError(status, msg.decode(errors="replace"))
