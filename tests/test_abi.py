"""The C ABI boundary without a GPU: the library builds for sm_103a, loads, and
exports every function that include/ozfft.h declares (no compute calls)."""
import ctypes
import os
import re

import pytest

from paper_2603_29129_gb300 import build, ozfft

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ozfft.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ozfft_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ctypes.CDLL(build.LIB)


def test_header_declares_the_boundary():
    names = declared_functions()
    assert {"ozfft_plan", "ozfft_execute", "ozfft_destroy"} <= set(names)
    assert sorted(ozfft.EXPORTS) == names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_loads_and_reports_errors_without_gpu(lib):
    L = ozfft.load(build.LIB)
    assert L.ozfft_error_string(ozfft.ERR_RANGE) == b"input magnitude out of range"
    assert L.ozfft_error_string(12345) == b"unknown error"
    # argument validation happens on the host before any device work
    assert L.ozfft_plan(0, 1, ozfft.FORWARD) is None
    assert b"argument" in L.ozfft_last_error()
    opt = ozfft.Options(3, 1, 2, 12, 0)   # N = 12 is not a power of two
    assert L.ozfft_plan_ex(8, 1, ozfft.FORWARD, ctypes.byref(opt)) is None
    assert b"power of two" in L.ozfft_last_error()
    assert L.ozfft_execute(None, None, None, None) == ozfft.ERR_ARG


def test_kernels_are_built_for_sm_103a():
    # the link step embeds sm_103a SASS; check the build flags rather than the binary
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.NVCC_FLAGS)


@pytest.mark.parametrize("value,expect", [
    (None, (ozfft.OK, 0, 0)),
    ("", (ozfft.OK, 0, 0)),
    ("alloc", (ozfft.OK, 1, 0)),
    ("alloc:3", (ozfft.OK, 1, 3)),
    ("status:6", (ozfft.OK, 2, 6)),
    ("status:8", (ozfft.OK, 2, 8)),
    ("alloc:0", (ozfft.ERR_ARG, 0, 0)),
    ("alloc:-1", (ozfft.ERR_ARG, 0, 0)),
    ("status:4", (ozfft.ERR_ARG, 0, 0)),     # not a device status code
    ("status:9", (ozfft.ERR_ARG, 0, 0)),
    ("bogus", (ozfft.ERR_ARG, 0, 0)),
])
def test_fault_hook_parsing_without_gpu(lib, monkeypatch, value, expect):
    """OZFFT_FAULT is parsed on the host: the settings the failure tests use and
    malformed ones, which are argument errors rather than silently ignored."""
    ozfft.load(build.LIB)
    if value is None:
        monkeypatch.delenv("OZFFT_FAULT", raising=False)
    else:
        monkeypatch.setenv("OZFFT_FAULT", value)
    assert ozfft.fault_config() == expect
    if expect[0] != ozfft.OK:
        assert b"OZFFT_FAULT" in ozfft.load().ozfft_last_error()


def test_plan_creation_rejects_bad_fault_setting_without_gpu(lib, monkeypatch):
    """A malformed OZFFT_FAULT stops plan creation on the host (before any
    device allocation) with the hook's message."""
    L = ozfft.load(build.LIB)
    monkeypatch.setenv("OZFFT_FAULT", "alloc:x")
    opt = ozfft.Options(3, 1, 2, 0, 0)
    assert L.ozfft_plan_ex(1024, 1, ozfft.FORWARD, ctypes.byref(opt)) is None
    assert b"OZFFT_FAULT" in L.ozfft_last_error()
