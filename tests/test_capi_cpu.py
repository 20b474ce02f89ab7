"""CPU checks of the C-ABI library: it builds for sm_103a, loads, and exports every
function the public header declares (no device calls: there may be no GPU)."""
import ctypes
import os
import re

import pytest

from paper_2105_10517_gb300 import gpspin

HEADER = os.path.join(gpspin.ROOT, "include", "gpspin.h")


def header_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gp_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    gpspin.build()
    return ctypes.CDLL(gpspin.LIB_PATH)


def test_header_declares_the_binding_exports():
    assert header_functions() == sorted(gpspin.EXPORTS)


def test_library_exports_every_header_symbol(lib):
    for name in header_functions():
        assert hasattr(lib, name), name


def test_strerror_needs_no_device(lib):
    lib.gp_strerror.restype = ctypes.c_char_p
    lib.gp_strerror.argtypes = [ctypes.c_int]
    assert lib.gp_strerror(0) == b"ok"
    assert b"invalid" in lib.gp_strerror(1)


def test_create_rejects_invalid_parameters_before_any_device_call(lib):
    lib = gpspin.load()
    h = ctypes.c_void_p()
    for bad in (dict(nx=3), dict(dt=0.0), dict(xlen=-1.0), dict(so_type=7), dict(c0=float("nan")), dict(precision=9)):
        p = dict(nx=16, ny=16, xlen=8.0, ylen=8.0, dt=0.01)
        p.update(bad)
        assert lib.gp_create(ctypes.byref(gpspin.make_params(p)), None, ctypes.byref(h)) == 1
    assert lib.gp_create(None, None, ctypes.byref(h)) == 1


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(gpspin, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(gpspin, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        gpspin.load()


def test_noalloc_rejects_before_any_device_work(lib):
    """gp_propagate_noalloc turns a misaligned psi pointer and a grid beyond its
    fixed scratch into errors before it touches the device (there is no device
    here: any CUDA call would fail with GP_ERR_CUDA instead)."""
    lib = gpspin.load()
    p = gpspin.make_params(dict(nx=64, ny=64, xlen=8.0, ylen=8.0, dt=0.01))
    misaligned = ctypes.c_void_p(0x1000 + 8)
    assert lib.gp_propagate_noalloc(ctypes.byref(p), misaligned, 1, 0, None) == 1
    big = gpspin.make_params(dict(nx=257, ny=16, xlen=8.0, ylen=8.0, dt=0.01))
    assert lib.gp_propagate_noalloc(ctypes.byref(big), ctypes.c_void_p(0x1000), 1, 0, None) == 6
    assert lib.gp_propagate_noalloc(ctypes.byref(p), None, 1, 0, None) == 1


def test_null_handles_are_rejected_without_a_device(lib):
    """The entry points added for the solve kind, the debug checks and the batched
    launch form check their arguments on the host first (GP_ERR_ARG = 1)."""
    lib = gpspin.load()
    assert lib.gp_set_debug(None, gpspin.DEBUG_POISON) == 1
    assert lib.gp_set_tiling(None, 0, 0, 1, 1, 32, 1) == 1
    assert lib.gp_batch_set_persistent(None, 0) == 1
    assert lib.gp_batch_use_graphs(None, 1) == 1

