"""The C-ABI library loads, exports every symbol its header declares, and
applies its host-side argument checks without touching a GPU."""
import ctypes
import os
import re

import pytest

from paper_1712_09789_gb300 import build as ccl_build
from paper_1712_09789_gb300 import ccl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_functions():
    names = []
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b([A-Za-z_][A-Za-z0-9_]*)\s*\(", text):
            name = m.group(1)
            if name.startswith("ccl_") and not name.endswith("_t"):
                names.append(name)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    ccl_build.build()
    return ccl.load()


def test_header_declares_the_entry_points():
    names = declared_functions()
    for must in ("ccl_label", "ccl_label_ws", "ccl_workspace_size", "ccl_label_host",
                 "ccl_get_device_status", "ccl_status_string"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    raw = ctypes.CDLL(ccl.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(raw, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_status_strings(lib):
    assert ccl.ccl_status_string(0) == "CCL_OK"
    assert ccl.ccl_status_string(5) == "CCL_ERR_DEVICE_TIMEOUT"
    assert ccl.ccl_status_string(999) == "CCL_ERR_UNKNOWN"
    assert ccl.ccl_version() >= 100


def test_workspace_size_host_logic(lib):
    assert ccl.ccl_workspace_size(0, 10) == 0
    a = ccl.ccl_workspace_size(64, 512)
    b = ccl.ccl_workspace_size(65, 513)  # four 512x64 blocks instead of one
    assert a > 0 and b > 3 * a
    # scratch stays below 2 bytes of address space per pixel
    assert ccl.ccl_workspace_size(8192, 8192) < 2 * 8192 * 8192
    with pytest.raises(ccl.CclError):
        ccl.ccl_workspace_size(-1, 5)
    with pytest.raises(ccl.CclError) as e:
        ccl.ccl_workspace_size(65536, 32768)  # H*W = 2^31 > 2^31 - 2
    assert e.value.status == ccl.CCL_ERR_UNSUPPORTED


def test_argument_checks_before_any_device_work(lib):
    f = lib.ccl_label
    dummy_in, dummy_out = 0x10000, 0x90000000
    # connectivity
    assert f(dummy_in, 4, 4, 4, 6, dummy_out, None) == ccl.CCL_ERR_INVALID_ARG
    # negative sizes
    assert f(dummy_in, -1, 4, 4, 8, dummy_out, None) == ccl.CCL_ERR_INVALID_ARG
    # pitch < W
    assert f(dummy_in, 4, 8, 4, 8, dummy_out, None) == ccl.CCL_ERR_INVALID_ARG
    # NULL pointers
    assert f(None, 4, 4, 4, 8, dummy_out, None) == ccl.CCL_ERR_INVALID_ARG
    assert f(dummy_in, 4, 4, 4, 8, None, None) == ccl.CCL_ERR_INVALID_ARG
    # too many pixels for int32 labels
    assert f(dummy_in, 65536, 32768, 65536, 8, dummy_out, None) == ccl.CCL_ERR_UNSUPPORTED
    # overlapping input and output
    assert f(dummy_in, 16, 16, 16, 8, dummy_in + 64, None) == ccl.CCL_ERR_INVALID_ARG
    # empty images are a no-op
    assert f(None, 0, 16, 16, 8, None, None) == ccl.CCL_OK
    assert f(None, 16, 0, 16, 4, None, None) == ccl.CCL_OK
    # caller-owned scratch must be present, aligned and large enough
    g = lib.ccl_label_ws
    assert g(dummy_in, 32, 32, 32, 8, dummy_out, None, 1 << 20, None) == ccl.CCL_ERR_INVALID_ARG
    assert g(dummy_in, 32, 32, 32, 8, dummy_out, 0x20000 + 8, 1 << 20, None) == ccl.CCL_ERR_INVALID_ARG
    assert g(dummy_in, 32, 32, 32, 8, dummy_out, 0x20000, 16, None) == ccl.CCL_ERR_INVALID_ARG


def test_variant_argument_checks(lib):
    # host-side checks only: a bad variant or connectivity is refused before
    # anything is launched
    assert lib.ccl_label_variant(None, 4, 4, 4, 8, 7, None, None, None) == ccl.CCL_ERR_INVALID_ARG
    assert lib.ccl_label_variant(None, 4, 4, 4, 5, 0, None, None, None) == ccl.CCL_ERR_INVALID_ARG
    assert lib.ccl_label_variant(None, 0, 4, 4, 8, 0, None, None, None) == ccl.CCL_OK


def test_component_stats_argument_checks(lib):
    n = ctypes.c_int(-1)
    assert lib.ccl_component_stats(None, -1, 4, None, 0, ctypes.byref(n), None) == ccl.CCL_ERR_INVALID_ARG
    assert lib.ccl_component_stats(None, 4, 4, None, 3, ctypes.byref(n), None) == ccl.CCL_ERR_INVALID_ARG
    assert lib.ccl_component_stats(None, 4, 4, None, 0, None, None) == ccl.CCL_ERR_INVALID_ARG
    assert lib.ccl_component_stats(None, 65536, 32768, None, 0, ctypes.byref(n), None) == ccl.CCL_ERR_UNSUPPORTED
    assert lib.ccl_component_stats(None, 0, 4, None, 0, ctypes.byref(n), None) == ccl.CCL_OK and n.value == 0


def test_volume_argument_checks(lib):
    # host-side checks only: every case below returns before a launch
    f = lib.ccl_label_3d
    vin, vout = 0x100000, 0x40000000
    for conn in (4, 8, 18, 0):
        assert f(vin, 2, 2, 2, 2, conn, vout, None) == ccl.CCL_ERR_INVALID_ARG
    assert f(vin, -1, 2, 2, 2, 6, vout, None) == ccl.CCL_ERR_INVALID_ARG
    assert f(vin, 2, 2, -2, 2, 26, vout, None) == ccl.CCL_ERR_INVALID_ARG
    assert f(None, 0, 5, 5, 5, 6, None, None) == ccl.CCL_OK
    assert f(None, 5, 5, 0, 5, 26, None, None) == ccl.CCL_OK
    assert f(None, 2, 2, 2, 2, 6, vout, None) == ccl.CCL_ERR_INVALID_ARG
    assert f(vin, 2, 2, 2, 2, 6, None, None) == ccl.CCL_ERR_INVALID_ARG
    assert f(vin, 2, 2, 4, 3, 6, vout, None) == ccl.CCL_ERR_INVALID_ARG          # pitch < W
    assert f(vin, 2048, 1024, 1024, 1024, 6, vout, None) == ccl.CCL_ERR_UNSUPPORTED
    assert f(vin, 4, 4, 4, 4, 26, vin + 8, None) == ccl.CCL_ERR_INVALID_ARG     # overlapping buffers
