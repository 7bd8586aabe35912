"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every function include/bpm.h declares, and rejects bad arguments before any
device work."""
import ctypes
import os

import pytest

from paper_1706_02261_b300 import build as build_mod


@pytest.fixture(scope="module")
def B():
    build_mod.build()
    from paper_1706_02261_b300 import bpm
    return bpm


def test_library_exports_every_declared_symbol(B):
    names = B.declared_symbols()
    assert {"bpm_plan", "bpm_propagate", "bpm_multiplex_psf", "bpm_free", "bpm_last_error",
            "bpm_check", "bpm_light_sheet"} <= set(names)
    lib = B.library()
    for name in names:
        assert hasattr(lib, name), name


def test_bad_arguments_rejected_without_device_work(B):
    lib = B.library()
    h = ctypes.c_void_p()
    assert lib.bpm_plan(ctypes.byref(h), None, 1, 0, None) == B.BPM_ERR_ARG
    d = (B.bpm_instance_desc * 1)(B.Instance(100, 4, 0.1, 0.1).desc())
    assert lib.bpm_plan(ctypes.byref(h), d, 1, 0, None) == B.BPM_ERR_UNSUPPORTED
    assert "not one of" in B.bpm_last_error()
    d = (B.bpm_instance_desc * 1)(B.Instance(1024, 4, 0.1, 0.1, ny=100).desc())
    assert lib.bpm_plan(ctypes.byref(h), d, 1, 0, None) == B.BPM_ERR_UNSUPPORTED
    # batched plans take square grids only
    d = (B.bpm_instance_desc * 2)(B.Instance(128, 4, 0.1, 0.1).desc(), B.Instance(128, 4, 0.1, 0.1, ny=256).desc())
    assert lib.bpm_plan(ctypes.byref(h), d, 2, 0, None) == B.BPM_ERR_UNSUPPORTED
    assert "square" in B.bpm_last_error()
    d = (B.bpm_instance_desc * 1)(B.Instance(64, 4, 0.0, 0.1).desc())
    assert lib.bpm_plan(ctypes.byref(h), d, 1, 0, None) == B.BPM_ERR_ARG
    d = (B.bpm_instance_desc * 1)(B.Instance(64, -1, 0.1, 0.1).desc())
    assert lib.bpm_plan(ctypes.byref(h), d, 1, 0, None) == B.BPM_ERR_ARG
    d = (B.bpm_instance_desc * 1)(B.Instance(64, 4, 0.1, 0.1).desc())
    assert lib.bpm_plan(ctypes.byref(h), d, 1, 0x100, None) == B.BPM_ERR_ARG
    assert lib.bpm_propagate(None, None, None, None, None, 0, 1, None) == B.BPM_ERR_ARG
    assert lib.bpm_free(None) == B.BPM_OK
    assert lib.bpm_check(None) == B.BPM_ERR_ARG


def test_library_is_built_for_sm103a(B):
    assert os.path.exists(B.LIB_PATH)
    assert "arch=compute_103a,code=sm_103a" in " ".join(build_mod.ARCH)
