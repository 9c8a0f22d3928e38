"""The C ABI library builds (nvcc cross-compiles for sm_103a without a GPU),
loads, and exports every function include/dms.h declares; host-side argument
checks answer without launching anything."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dms.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(?:int|int64_t|size_t|const char\s*\*)\s+(dms_\w+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2505_21266_gb300 import _lib
    return _lib.load()


def test_header_declares_the_four_calls():
    names = declared_functions()
    for n in ("dms_order", "dms_gradient", "dms_critical", "dms_diagram_d0d2"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2505_21266_gb300 import _lib
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.library_path()],
                         capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (dms_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    bound = {name for name, _, _ in _lib.SIGNATURES}
    assert set(declared_functions()) <= bound


def test_host_side_validation(lib):
    from paper_2505_21266_gb300 import _lib
    bad = _lib.dms_dims(1, 4, 4)
    good = _lib.dms_dims(4, 4, 4)
    assert lib.dms_num_vertices(bad) == 0
    assert lib.dms_num_vertices(good) == 64
    assert lib.dms_num_vertices(_lib.dms_dims(65536, 65536, 2)) == 0  # >= 2^32 - 1
    # errors found on the host come back before any CUDA call
    assert lib.dms_order(None, bad, None, None, 0, None, None) == 2
    assert lib.dms_order(None, good, None, None, 0, None, None) == 1
    fake = ctypes.c_void_p(0x1000)
    assert lib.dms_order(fake, good, fake, fake, 16, fake, None) == 5  # workspace too small
    assert lib.dms_gradient(None, good, None, None, None, None) == 1
    for code in range(10):
        assert lib.dms_status_string(code)
    assert lib.dms_order_workspace_size(good) > 0
