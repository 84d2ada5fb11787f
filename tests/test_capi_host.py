"""CPU-only checks of the C ABI: the library builds and loads, exports every
entry point that include/*.h declares, and rejects invalid input with the
documented status without touching a GPU (and reports ECUDA, not a
fallback, when there is no device)."""
import ctypes as C
import glob
import os
import re

import numpy as np
import pytest

import geometry as G

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def capi():
    from paper_2408_06880_gb300 import build as B
    B.build()
    from paper_2408_06880_gb300 import _capi
    return _capi


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:slbm_status|void|const char\s*\*)\s*\*?\s*(\w+)\s*\(", text, re.M):
            names.add(m.group(1))
    return names


def test_every_declared_symbol_is_exported(capi):
    names = declared_functions()
    assert len(names) >= 20
    L = C.CDLL(capi.LIB_PATH)
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    # and the binding declares exactly the header's entry points
    assert names == set(capi.SIGNATURES)


def _desc(capi, flags, **kw):
    d = capi.Desc()
    nz, ny, nx = flags.shape
    d.nx, d.ny, d.nz = nx, ny, nz
    d.flags = flags.ctypes.data
    d.periodic, d.q, d.op = 7, 19, capi.SRT
    d.omega_plus, d.trt_magic = 1.25, 3 / 16
    d.rho_out, d.storage, d.layout = 1.0, capi.FP32, capi.SPARSE
    for k, v in kw.items():
        setattr(d, k, v)
    return d


@pytest.mark.parametrize("field,value", [
    ("nx", 0), ("q", 15), ("op", 5), ("op", -1), ("omega_plus", 0.0), ("omega_plus", 2.0), ("storage", 3),
    ("scale_exp", 41), ("layout", 3), ("order", 3), ("trt_magic", -1.0), ("rho_out", 0.0),
])
def test_invalid_descriptors_are_rejected(capi, field, value):
    flags = np.zeros((4, 4, 4), np.uint8)
    d = _desc(capi, flags, **{field: value})
    if field == "trt_magic":
        d.op = capi.TRT
    h = C.c_void_p()
    st = capi.lib().sparse_lbm_create(C.byref(d), None, None, C.byref(h))
    assert st == capi.EINVAL
    assert h.value is None
    assert capi.lib().sparse_lbm_last_error()


def test_bad_flags_and_inlet_count(capi):
    flags = np.zeros((4, 4, 4), np.uint8)
    flags[0, 0, 0] = 9
    h = C.c_void_p()
    assert capi.lib().sparse_lbm_create(C.byref(_desc(capi, flags)), None, None, C.byref(h)) == capi.EINVAL
    flags[0, 0, 0] = 2
    u = np.zeros((2, 3), np.float32)
    d = _desc(capi, flags, inlet_u=u.ctypes.data, n_inlet_u=2)
    assert capi.lib().sparse_lbm_create(C.byref(d), None, None, C.byref(h)) == capi.EINVAL
    d = _desc(capi, flags, layout=capi.DENSE)
    assert capi.lib().sparse_lbm_create(C.byref(d), None, None, C.byref(h)) == capi.EUNSUPPORTED
    # MRT is D3Q19 only, the central-moment and cumulant operators D3Q27 only
    for q, op in ((27, capi.MRT), (19, capi.CM), (19, capi.CUMULANT)):
        d = _desc(capi, np.zeros((4, 4, 4), np.uint8), q=q, op=op)
        assert capi.lib().sparse_lbm_create(C.byref(d), None, None, C.byref(h)) == capi.EUNSUPPORTED
    for op in (capi.CM, capi.CUMULANT):
        d = _desc(capi, np.zeros((4, 4, 4), np.uint8), q=27, op=op, layout=capi.DENSE)
        assert capi.lib().sparse_lbm_create(C.byref(d), None, None, C.byref(h)) == capi.EUNSUPPORTED


def test_no_device_means_ecuda_not_fallback(capi):
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    flags = G.relaxed_spheres().flags
    h = C.c_void_p()
    st = capi.lib().sparse_lbm_create(C.byref(_desc(capi, flags)), None, None, C.byref(h))
    assert st == capi.ECUDA
    assert b"no CUDA device" in capi.lib().sparse_lbm_last_error()


def test_null_arguments(capi):
    L = capi.lib()
    assert L.sparse_lbm_step(None, 1) == capi.EINVAL
    assert L.sparse_lbm_reduce(None, None, 1) == capi.EINVAL
    L.sparse_lbm_free(None)      # no-op
    h = C.c_void_p()
    assert L.sparse_lbm_create(None, None, None, C.byref(h)) == capi.EINVAL
