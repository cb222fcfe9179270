"""Host-side checks of the C ABI that need no GPU: the library builds, loads, exports
every entry point include/sse.h declares, and rejects bad arguments with codes."""
import ctypes
import os
import re

import pytest

from paper_1912_08810_gb300 import build as sse_build
from paper_1912_08810_gb300 import sse

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"SSE_API\s+[\w\s\*]+?\b(sse_\w+)\s*\(", src)
    return names


@pytest.fixture(scope="module")
def lib():
    sse_build.build()
    return sse.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_entry_points()
    assert len(names) >= 9
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(sse.EXPORTED)


def test_status_strings(lib):
    assert sse.sse_status_string(0) == "SSE_OK"
    assert sse.sse_status_string(-5) == "SSE_E_TIMEOUT"
    assert sse.sse_status_string(1234) == "SSE_E_UNKNOWN_STATUS"
    assert sse.sse_abi_version() == 1


def test_null_arguments_are_rejected(lib):
    h = ctypes.c_void_p()
    assert lib.sse_plan(None, ctypes.byref(h)) == sse.SSE_E_INVALID_ARG
    assert "NULL" in sse.sse_last_error()
    assert lib.sse_plan(ctypes.byref(sse.sse_geometry()), None) == sse.SSE_E_INVALID_ARG
    assert lib.sse_execute(None, None, None) == sse.SSE_E_INVALID_ARG
    assert lib.sse_plan_query(None, None) == sse.SSE_E_INVALID_ARG
    assert lib.sse_plan_destroy(None) == sse.SSE_OK


@pytest.mark.parametrize("field,value,msg", [
    ("nkz", 0, "positive"), ("ne", -3, "positive"), ("norb", 10, "norb"),
    ("omega_first", -(1 << 20), "omega_first"), ("dtype", 7, "dtype"), ("mode", 5, "mode"),
])
def test_bad_geometry_rejected_before_any_device_call(lib, field, value, msg):
    g = sse.sse_geometry(3, 3, 8, 2, 4, 2, 12, 1, None, None, 0, 0)
    setattr(g, field, value)
    h = ctypes.c_void_p()
    assert lib.sse_plan(ctypes.byref(g), ctypes.byref(h)) == sse.SSE_E_INVALID_ARG
    assert msg in sse.sse_last_error()
    assert not h.value


def test_debug_inject_checks_its_argument(lib):
    assert lib.sse_debug_inject(99) == sse.SSE_E_INVALID_ARG
    assert "injection" in sse.sse_last_error()
    assert lib.sse_debug_inject(sse.SSE_INJECT_ALLOC_FAIL) == sse.SSE_OK
    assert lib.sse_debug_inject(sse.SSE_INJECT_NONE) == sse.SSE_OK  # disarmed again


def test_server_entry_points_reject_null(lib):
    assert lib.sse_server_shutdown(None) == sse.SSE_E_INVALID_ARG
    assert lib.sse_server_destroy(None) == sse.SSE_OK
    assert lib.sse_poll(None, 1, None) == sse.SSE_E_INVALID_ARG
