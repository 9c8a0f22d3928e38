"""The gradient kernel's ProcessLowerStars (paper_2505_21266_gb300/csrc/
dms_lowerstar.cuh, which also compiles for the host) against the oracle on
the CPU: every discrete vector and critical simplex of small grids with
ties, plateaus and noise, bit for bit.  This pins the kernel's restatement
of the algorithm (PQone's triangles drained before its tets, a triangle
moved to PQzero when its last edge is classified) without a GPU; the GPU
parity tests check the kernel itself."""
import ctypes
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
import record_decode as rd

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2505_21266_gb300", "csrc")


@pytest.fixture(scope="module")
def host_lib():
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tempfile.mkdtemp(prefix="dms_host_ls_")
    so = os.path.join(d, "host_lowerstar.so")
    subprocess.run([cxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-I", CSRC,
                    os.path.join(HERE, "host_lowerstar.cpp"), "-o", so], check=True)
    lib = ctypes.CDLL(so)
    lib.host_gradient.restype = ctypes.c_int
    yield lib
    shutil.rmtree(d, ignore_errors=True)


def _check(lib, f):
    f = np.ascontiguousarray(f, dtype=np.float32)
    nz, ny, nx = f.shape
    r = oracle.run(f, diagrams=False)
    order = r.order.astype(np.uint32)
    desc = np.zeros(f.size, np.uint8)
    rec = np.zeros(f.size, np.uint64)
    assert lib.host_gradient(order.ctypes.data, nx, ny, nz, desc.ctypes.data, rec.ctypes.data) == 0
    pairs, crit = rd.decode(desc, rec, nx, ny, nz)
    assert np.array_equal(pairs, r.get(oracle.GRAD_PAIRS))
    for d in range(4):
        assert np.array_equal(crit[d], r.crit(d)), d


def test_host_lower_star_random_small(host_lib):
    rng = np.random.default_rng(20)
    for it in range(120):
        shape = tuple(int(x) for x in rng.integers(2, 8, size=3))
        levels = int(rng.integers(2, 5)) if it % 2 else 1 << 20
        _check(host_lib, rng.integers(0, levels, size=shape).astype(np.float32))


def test_host_lower_star_fields(host_lib):
    from paper_2505_21266_gb300 import fields
    _check(host_lib, fields.gaussian_mixture((20, 22, 24), 8, (0.05, 0.2), 1e-3, 1).numpy())
    _check(host_lib, fields.quantized_noise((18, 19, 20), 256, 3).numpy())
    _check(host_lib, fields.uniform01((16, 17, 18), 4).numpy())


def test_host_lower_star_hand_worked_cases(host_lib):
    """The kernel's restated pop order on the lower stars worked by hand from
    the algorithm (tests/golden/lower_stars.json)."""
    import refcomplex as rc
    from test_oracle_pins import golden_lower_stars
    cx = rc.Complex(3, 3, 3)
    for name, f, x, exp_pairs, exp_crit in golden_lower_stars():
        order = rc.canonical_order(f).astype(np.uint32)
        desc = np.zeros(27, np.uint8)
        rec = np.zeros(27, np.uint64)
        assert lib_ok(host_lib, order, desc, rec)
        pairs, crit = rd.decode(desc, rec, 3, 3, 3)
        got = {tuple(int(v) for v in p) for p in pairs
               if cx.max_vertex(cx.verts(int(p[0]), int(p[1])), order) == x}
        assert got == exp_pairs, name
        got_c = {(d, int(i)) for d in range(4) for i in crit[d]
                 if cx.max_vertex(cx.verts(d, int(i)), order) == x}
        assert got_c == exp_crit, name


def lib_ok(lib, order, desc, rec):
    return lib.host_gradient(order.ctypes.data, 3, 3, 3, desc.ctypes.data, rec.ctypes.data) == 0
