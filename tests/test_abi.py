"""CPU-side checks of the C ABI: the CUDA library builds for sm_103a, loads, exports
every function include/ccl.h declares, and rejects bad arguments before touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w\s\*]*?\b(ccl_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import paper_1606_05973_gb300 as ccl

    ccl.build()
    return ctypes.CDLL(ccl.build())


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("ccl_label", "ccl_label_async", "ccl_label_host", "ccl_label_batch",
                 "ccl_status_string", "ccl_profile_read"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert missing == []


def test_checked_build_exports_too():
    import paper_1606_05973_gb300 as ccl

    dbg = ctypes.CDLL(ccl.build(debug=True))
    assert [n for n in declared_functions() if not hasattr(dbg, n)] == []


def test_status_strings_and_version(lib):
    lib.ccl_status_string.restype = ctypes.c_char_p
    assert lib.ccl_status_string(0) == b"ok"
    assert b"unsupported" in lib.ccl_status_string(2)
    assert lib.ccl_version() >= 100


def test_argument_checks_need_no_gpu(lib):
    k = ctypes.c_int32(0)
    p = ctypes.c_void_p(16)  # never dereferenced: the checks fail first
    assert lib.ccl_label(p, -1, 4, 4, 8, p, ctypes.byref(k), None) == 1
    assert lib.ccl_label(p, 4, 4, 3, 8, p, ctypes.byref(k), None) == 1
    assert lib.ccl_label(None, 4, 4, 4, 8, p, ctypes.byref(k), None) == 1
    assert lib.ccl_label(p, 4, 4, 3, 4, p, ctypes.byref(k), None) == 1  # 4-connectivity: same checks
    assert lib.ccl_label(p, 4, 4, 4, 5, p, ctypes.byref(k), None) == 2  # connectivity: UNSUPPORTED
    assert lib.ccl_label(p, 0, 9, 9, 5, p, ctypes.byref(k), None) == 2  # connectivity checked first
    assert lib.ccl_label(p, -1, 4, 4, 6, p, ctypes.byref(k), None) == 2
    for conn in (8, 4):
        k.value = 7
        assert lib.ccl_label(p, 0, 9, 9, conn, p, ctypes.byref(k), None) == 0 and k.value == 0
    for t in (-1, 256):  # threshold outside a byte's range
        assert lib.ccl_label_threshold(p, 4, 4, 4, 8, t, p, ctypes.byref(k), None) == 1
    assert lib.ccl_label_threshold(p, 0, 9, 9, 8, 127, p, ctypes.byref(k), None) == 0 and k.value == 0
    # process-wide options: checked on the host, no GPU call (restored to the defaults)
    for bad in (-1, 4):
        assert lib.ccl_set_tile_policy(bad) == 1
    for ok in (1, 2, 0):
        assert lib.ccl_set_tile_policy(ok) == 0
    assert lib.ccl_set_global_ctas_per_sm(-1) == 1
    assert lib.ccl_set_launch_mode(4) == 1 and lib.ccl_set_launch_mode(-1) == 1
    assert lib.ccl_set_tuning(None, 1, 300, 700, 64, 0) == 1  # rows missing
    assert lib.ccl_set_tuning(None, 0, 0, 0, 0, 0) == 0       # back to the built-in table
    assert lib.ccl_set_global_ctas_per_sm(1) == 0 and lib.ccl_set_global_ctas_per_sm(0) == 0
    nb = ctypes.c_int64(0)
    assert lib.ccl_workspace_bytes(8192, 8192, ctypes.byref(nb)) == 0
    # the largest layout over the modes.  8-connectivity: bit pack 1/8 B/px + run codes
    # 1/2 B/px + parents (row segments) 2 B/px + edge ids + segment counts, under 3 B/px;
    # 4-connectivity: one-row strips double the run-code slots (1 B/px) and 32-row tiles
    # the row-edge ids (about 3.4 B/px); multi-class: runs of different classes may touch,
    # so run codes (2 B/px) and parents (4 B/px) double again, plus the run-start bit pack
    assert 6.3 * 8192 * 8192 < nb.value < 6.8 * 8192 * 8192
