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
    names = re.findall(r"\b(?:int|int32_t|int64_t|size_t|const char\s*\*)\s+(dms_\w+)\s*\(", text)
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


def test_batch_host_validation(lib):
    from paper_2505_21266_gb300 import _lib
    assert lib.dms_batch_tile_variants() == 6
    assert lib.dms_batch_max_rounds() > 0
    T = _lib.dms_field_desc * 2
    good = T(_lib.dms_field_desc(0, 4, 5, 6, 0), _lib.dms_field_desc(120, 3, 3, 3, 0))
    gap = T(_lib.dms_field_desc(0, 4, 5, 6, 0), _lib.dms_field_desc(121, 3, 3, 3, 0))
    thin = T(_lib.dms_field_desc(0, 4, 5, 6, 0), _lib.dms_field_desc(120, 1, 3, 3, 0))
    caps = (ctypes.c_int64 * 4)(10, 10, 10, 10)
    assert lib.dms_batch_workspace_size(ctypes.byref(good), 2, caps, 10) > 0
    assert lib.dms_batch_workspace_size(ctypes.byref(gap), 2, caps, 10) == 0
    assert lib.dms_batch_workspace_size(ctypes.byref(thin), 2, caps, 10) == 0
    assert lib.dms_batch_workspace_size(ctypes.byref(good), 0, caps, 10) == 0
    neg = (ctypes.c_int64 * 4)(10, -1, 10, 10)
    assert lib.dms_batch_workspace_size(ctypes.byref(good), 2, neg, 10) == 0
    fake = ctypes.c_void_p(0x1000)
    args = lambda table, variant, wsb: lib.dms_batch_diagrams(
        fake, ctypes.byref(table), fake, 2, variant, fake, fake, fake, caps, 10, fake, fake, fake,
        fake, fake, fake, wsb, fake, None)
    assert args(gap, 0, 1 << 40) == 8     # DMS_ERR_ARG: offsets not contiguous
    assert args(thin, 0, 1 << 40) == 2    # DMS_ERR_DIMS
    assert args(good, 6, 1 << 40) == 8    # no such tile variant
    assert args(good, 0, 16) == 5         # DMS_ERR_WORKSPACE


def test_diagram_workspace_size_covers_its_parts(lib):
    """The D0/D2 workspace holds, at least, one claim word per tetrahedron
    id and, per saddle, its 32-byte record plus three 4-byte list entries
    (two live lists and the spanning-forest list); it grows with the
    saddle and extremum counts."""
    from paper_2505_21266_gb300 import _lib
    d = _lib.dms_dims(40, 50, 60)
    n = 40 * 50 * 60

    def size(c0, c1, c2, c3):
        return lib.dms_diagram_workspace_size(d, (ctypes.c_int64 * 4)(c0, c1, c2, c3))

    base = size(10, 100, 100, 10)
    assert base >= 24 * n + 44 * 100
    assert size(10, 100_000, 100, 10) - base >= 44 * (100_000 - 100)
    assert size(10, 100, 100_000, 10) - base >= 44 * (100_000 - 100)
    assert size(50_000, 100, 100, 10) > base  # union-find nodes


def test_d1_and_selfcorrecting_host_validation(lib):
    """The D1 call and the self-correcting D0/D2 call answer bad arguments on
    the host, before any launch; the D1 workspace grows with its pool."""
    from paper_2505_21266_gb300 import _lib
    d = _lib.dms_dims(8, 9, 10)
    nc = (ctypes.c_int64 * 4)(5, 50, 40, 4)
    w0 = lib.dms_diagram_d1_workspace_size(d, nc, 0)
    assert w0 > 0
    assert lib.dms_diagram_d1_workspace_size(d, nc, 10 * w0) > w0
    assert lib.dms_diagram_d1_workspace_size(_lib.dms_dims(1, 9, 10), nc, 0) == 0
    fake = ctypes.c_void_p(0x1000)
    call = lambda dims, ncrit, d0n, cap, pool, wsb: lib.dms_diagram_d1(
        fake, fake, fake, dims, fake, fake, ncrit, fake, d0n, fake, 0, fake, cap, fake, pool,
        fake, wsb, fake, None)
    assert call(_lib.dms_dims(1, 9, 10), nc, 0, 40, 0, 1 << 40) == 2   # DMS_ERR_DIMS
    assert call(d, nc, -1, 40, 0, 1 << 40) == 8                         # negative D0 count
    assert call(d, nc, 0, -1, 0, 1 << 40) == 8                          # negative capacity
    assert call(d, nc, 0, 40, -5, 1 << 40) == 8                         # negative pool
    assert call(d, nc, 0, 40, 0, 16) == 5                               # DMS_ERR_WORKSPACE
    assert lib.dms_diagram_d1(fake, None, fake, d, fake, fake, nc, fake, 0, fake, 0, fake, 40,
                              fake, 0, fake, 1 << 40, fake, None) == 1  # DMS_ERR_NULL
    sc = lambda dims, ncrit: lib.dms_diagram_d0d2_selfcorrecting(
        fake, fake, fake, fake, dims, fake, fake, fake, fake, ncrit, fake, 4, fake, 4, fake, fake,
        fake, 16, fake, None)
    assert sc(_lib.dms_dims(1, 9, 10), nc) == 2
    assert sc(d, (ctypes.c_int64 * 4)(0, 50, 40, 4)) == 8                 # no minimum
    assert sc(d, nc) == 5                                                  # workspace too small
