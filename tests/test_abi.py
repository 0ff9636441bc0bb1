"""The C-ABI library builds, loads without a GPU and exports every entry point
that include/mpbp.h declares (no compute calls here)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mpbp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mpbp_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("no CUDA toolkit")
    from paper_2312_14907_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_hot_path_calls():
    names = _declared()
    for n in ("mpbp_object_build", "mpbp_forward", "mpbp_loss_grad", "mpbp_step", "mpbp_create",
              "mpbp_set_data", "mpbp_set_probe", "mpbp_loss_grad_batched", "mpbp_loss_grad_host"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_export():
    from paper_2312_14907_gb300 import mpbp
    assert sorted(mpbp.EXPORTS) == _declared()


def test_status_strings_without_gpu(lib):
    lib.mpbp_status_string.restype = ctypes.c_char_p
    assert lib.mpbp_status_string(0) == b"MPBP_OK"
    assert lib.mpbp_status_string(6) == b"MPBP_ERR_BOUNDS"
    assert lib.mpbp_status_string(99) == b"MPBP_ERR_UNKNOWN"


def test_invalid_geometry_is_rejected_on_the_host(lib):
    from paper_2312_14907_gb300 import mpbp
    import numpy as np
    G = np.zeros((2, 3))
    scan = np.zeros((1, 2), np.int32)
    h = ctypes.c_void_p()
    bad_m = mpbp._Problem(16, 16, 3, 2, 24, 1, G.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                          scan.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), 0, 6.28)
    lib.mpbp_create.restype = ctypes.c_int
    assert lib.mpbp_create(ctypes.byref(bad_m), ctypes.byref(h)) == 2      # unsupported M
    bad_d = mpbp._Problem(16, 16, 3, 0, 16, 1, G.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                          scan.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), 0, 6.28)
    assert lib.mpbp_create(ctypes.byref(bad_d), ctypes.byref(h)) == 1      # no peaks
    assert h.value is None


def test_probe_shift_arguments_are_checked_on_the_host(lib):
    """mpbp_shift_probe validates sizes and offsets before any device call."""
    import numpy as np
    V = ctypes.c_void_p
    lib.mpbp_shift_probe.argtypes = [V, ctypes.c_int32, V, ctypes.c_int32, V, V]
    lib.mpbp_shift_probe.restype = ctypes.c_int
    d = np.zeros((2, 2))
    fake = ctypes.c_void_p(16)   # never dereferenced: every call below fails its checks first
    assert lib.mpbp_shift_probe(None, 8, d.ctypes.data, 2, fake, None) == 1
    assert lib.mpbp_shift_probe(fake, 0, d.ctypes.data, 2, fake, None) == 1
    assert lib.mpbp_shift_probe(fake, 129, d.ctypes.data, 2, fake, None) == 1
    assert lib.mpbp_shift_probe(fake, 8, d.ctypes.data, -1, fake, None) == 1
    for bad in (0.5000001, -0.75, np.nan, np.inf):
        d[1, 0] = bad
        assert lib.mpbp_shift_probe(fake, 8, d.ctypes.data, 2, fake, None) == 1
    d[1, 0] = 0.5
    assert lib.mpbp_shift_probe(fake, 8, d.ctypes.data, 0, fake, None) == 0   # nothing to do
    lib.mpbp_set_scan_offsets.argtypes = [V, V, V]
    lib.mpbp_set_scan_offsets.restype = ctypes.c_int
    assert lib.mpbp_set_scan_offsets(None, d.ctypes.data, None) == 1
