"""libsop.so builds, loads and exports every entry point include/sop.h
declares; argument checks that run before any CUDA call (CPU only)."""
import ctypes
import os
import re

import pytest

from paper_1012_3911_gb300 import build as sop_build
from paper_1012_3911_gb300 import sop

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    sop_build.build()
    return sop.load()


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(sop_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("sop_plan_create", "sop_plan_destroy", "sop_bind_state", "sop_set_potential", "sop_step",
                     "sop_norm", "sop_energy", "sop_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_version_and_empty_error(lib):
    assert sop.sop_version() >= 1
    assert isinstance(sop.sop_last_error(), str)


@pytest.mark.parametrize("dims,comps,status", [
    ((7,), 1, sop.SOP_EUNSUPPORTED),       # below 8 and not 2^a 3^b
    ((40, 16), 1, sop.SOP_EUNSUPPORTED),   # factor 5
    ((18, 16), 1, sop.SOP_EUNSUPPORTED),   # 9 = 3^2 needs two radix-3 stages
    ((8192,), 1, sop.SOP_EUNSUPPORTED),    # above 4096
    ((16, 16, 16, 16), 1, sop.SOP_EINVAL), # ndim 4
    ((16, 16), 3, sop.SOP_EINVAL),         # components must be 1, 2 or 4
    ((16, 16), 2, sop.SOP_EUNSUPPORTED),   # two-component Dirac needs ndim = 1
    ((16,), 4, sop.SOP_EUNSUPPORTED),      # four-component Dirac needs ndim = 2 or 3
    ((16, 16, 16), 2, sop.SOP_EUNSUPPORTED),
])
def test_create_rejects_before_touching_the_gpu(lib, dims, comps, status):
    out = ctypes.c_void_p()
    nd = len(dims)
    cd = (ctypes.c_int64 * nd)(*dims)
    cs = (ctypes.c_double * nd)(*([0.1] * nd))
    rc = lib.sop_plan_create(ctypes.byref(out), nd, cd, cs, comps, sop.SOP_C64, None, None)
    assert rc == status
    assert out.value is None
    assert sop.sop_last_error() != ""


def test_null_arguments(lib):
    assert lib.sop_plan_create(None, 1, None, None, 1, 0, None, None) == sop.SOP_EINVAL
    assert lib.sop_bind_state(None, None) == sop.SOP_EINVAL
    assert lib.sop_step(None, 1, 0.1, None) == sop.SOP_EINVAL
    assert lib.sop_norm(None, None) == sop.SOP_EINVAL
    assert lib.sop_plan_destroy(None) == sop.SOP_OK
    out = ctypes.c_void_p()
    cd = (ctypes.c_int64 * 1)(16)
    cs = (ctypes.c_double * 1)(-1.0)
    assert lib.sop_plan_create(ctypes.byref(out), 1, cd, cs, 1, 0, None, None) == sop.SOP_EINVAL
    assert lib.sop_plan_create(ctypes.byref(out), 1, cd, (ctypes.c_double * 1)(0.1), 1, 7, None, None) == sop.SOP_EINVAL


def test_pass_shape_calls_reject_bad_arguments(lib):
    lib.sop_set_pass_shape.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
    lib.sop_autotune.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_void_p]
    assert lib.sop_set_pass_shape(None, 0, 0) == sop.SOP_EINVAL
    assert lib.sop_autotune(None, 0.1, 4, None) == sop.SOP_EINVAL
    assert sop.SOP_PASS_SHAPES == 8


def test_noalloc_wrapper_rejects_unsafe_tensors():
    """The Python wrapper checks tensors before the kernel could read or
    write out of bounds (no GPU call is made for a rejected argument)."""
    import torch
    cpu = torch.zeros(16, dtype=torch.complex64)
    out = torch.zeros(1, dtype=torch.float64)
    with pytest.raises(ValueError):
        sop.sop_norm_noalloc(cpu, 16, sop.SOP_C64, 1.0, out)   # not a CUDA tensor


def test_canary_check_is_a_check_build_entry_point():
    """sop_debug_check_canaries answers SOP_EUNSUPPORTED in a normal build
    (no GPU call) and rejects a null output pointer."""
    import os
    if os.environ.get("SOP_CHECK", "") == "1":
        pytest.skip("check build selected")
    lib = sop.load()
    lib.sop_debug_check_canaries.argtypes = [ctypes.c_void_p]
    lib.sop_debug_check_canaries.restype = ctypes.c_int
    assert lib.sop_debug_check_canaries(None) == sop.SOP_EINVAL
    with pytest.raises(sop.SopError) as ei:
        sop.sop_debug_check_canaries()
    assert ei.value.status == sop.SOP_EUNSUPPORTED
