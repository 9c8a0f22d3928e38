"""DMS oracle -- test infrastructure only.

A ctypes front end to ``dms_oracle.cpp``: a plain single-threaded CPU
restatement of the Discrete Morse Sandwich hot path (Distributed DMS, arXiv
2505.21266) -- the global vertex order (Sec. 2.1, Sec. 3), Robins' lower-star
discrete gradient (Sec. 2.3), the critical simplices ("zero-persistence skip",
Sec. 2.5) and the D0/D2 pairs of Alg. 1 and its dual (Sec. 2.5) -- plus a full
boundary-matrix reduction for small grids.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  It shares
no code with the CUDA library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dms_oracle.cpp")
_SRC2 = os.path.join(_HERE, "dms_oracle2d.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libdms_oracle.so")
_lock = threading.Lock()
_lib = None

# output selectors (mirror the enum in dms_oracle.cpp)
ORDER, CRIT0, CRIT1, CRIT2, CRIT3, GRAD_PAIRS, D0, D2, D0_ESSENTIAL = range(9)
D0_TRIPLETS, D2_TRIPLETS, PARTNER0, PARTNER1, PARTNER2, PARTNER3, REDUCTION = range(9, 16)
D1 = 16
RUN_ORDER, RUN_GRADIENT, RUN_DIAGRAMS, RUN_REDUCTION, RUN_D1 = 1, 2, 4, 8, 16

ABSENT = -2
CRITICAL = -1
OUTSIDE = -1

PAIR_DTYPE = np.dtype([("birth_id", "<i8"), ("death_id", "<i8"), ("birth", "<f4"),
                       ("death", "<f4"), ("birth_vtx", "<u4"), ("death_vtx", "<u4")])


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (plain C++17, -O2, no OpenMP)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC), os.path.getmtime(_SRC2))):
            return _LIB
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread", _SRC, _SRC2,
                               "-o", tmp])
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i64, vp = ctypes.c_int64, ctypes.c_void_p
        lib.orc_run.restype = vp
        lib.orc_run.argtypes = [vp, i64, i64, i64, ctypes.c_int]
        lib.orc_run_threads.restype = vp
        lib.orc_run_threads.argtypes = [vp, i64, i64, i64, ctypes.c_int, ctypes.c_int]
        lib.orc_status.restype = ctypes.c_int
        lib.orc_status.argtypes = [vp]
        lib.orc_count.restype = i64
        lib.orc_count.argtypes = [vp, ctypes.c_int]
        lib.orc_copy.restype = None
        lib.orc_copy.argtypes = [vp, ctypes.c_int, vp]
        lib.orc_free.restype = None
        lib.orc_free.argtypes = [vp]
        lib.orc_pair_extrema_saddles.restype = None
        lib.orc_pair_extrema_saddles.argtypes = [i64, vp, vp, i64, vp, vp]
        lib.orc_lower_star_vertex.restype = ctypes.c_int
        lib.orc_lower_star_vertex.argtypes = [vp, i64, i64, i64, i64, vp, i64, vp, vp, i64, vp]
        lib.orc2_run.restype = vp
        lib.orc2_run.argtypes = [vp, i64, i64, ctypes.c_int]
        lib.orc2_status.restype = ctypes.c_int
        lib.orc2_status.argtypes = [vp]
        lib.orc2_count.restype = i64
        lib.orc2_count.argtypes = [vp, ctypes.c_int]
        lib.orc2_copy.restype = None
        lib.orc2_copy.argtypes = [vp, ctypes.c_int, vp]
        lib.orc2_free.restype = None
        lib.orc2_free.argtypes = [vp]
        for name in ("orc_d0_edge_local", "orc_d2_triangle_local"):
            fn = getattr(lib, name)
            fn.restype = ctypes.c_int
            fn.argtypes = [vp, i64, i64, i64, i64, i64, vp]
        _lib = lib
    return _lib


class OracleError(RuntimeError):
    pass


_STATUS = {2: "bad dims (each >= 2, fewer than 2^32 - 1 vertices)", 3: "NaN in the field",
           90: "a simplex was left unclassified", 91: "a simplex was classified twice",
           92: "D1: the highest edge of a boundary is paired with a vertex",
           93: "D1: the highest edge of a boundary is a D0 death"}

_DTYPES = {ORDER: np.uint32, D0: PAIR_DTYPE, D2: PAIR_DTYPE, D0_ESSENTIAL: PAIR_DTYPE,
           D1: PAIR_DTYPE}


class Result:
    """Everything the oracle computed for one field (kept in C++ memory)."""

    def __init__(self, field: np.ndarray, flags: int, threads: int = 1):
        f = np.ascontiguousarray(field, dtype=np.float32)
        if f.ndim != 3:
            raise ValueError("field must be 3D, indexed [z, y, x]")
        self.nz, self.ny, self.nx = f.shape
        lib = _load()
        self._h = lib.orc_run_threads(f.ctypes.data, self.nx, self.ny, self.nz, flags,
                                      int(threads))
        st = lib.orc_status(self._h)
        if st:
            lib.orc_free(self._h)
            self._h = None
            raise OracleError(_STATUS.get(st, f"status {st}"))

    def get(self, what: int) -> np.ndarray:
        lib = _load()
        n = lib.orc_count(self._h, what)
        dt = _DTYPES.get(what, np.int64)
        out = np.empty(max(n, 0), dtype=dt)
        if n > 0:
            lib.orc_copy(self._h, what, out.ctypes.data)
        if what in (GRAD_PAIRS, D0_TRIPLETS, D2_TRIPLETS):
            out = out.reshape(-1, 3)
        if what == REDUCTION:
            out = out.reshape(-1, 3)
        return out

    @property
    def order(self):
        return self.get(ORDER)

    def crit(self, d: int) -> np.ndarray:
        return self.get(CRIT0 + d)

    def partner(self, d: int) -> np.ndarray:
        return self.get(PARTNER0 + d)

    def __del__(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.orc_free(self._h)
            self._h = None


def run(field: np.ndarray, order=True, gradient=True, diagrams=True, reduction=False,
        threads: int = 1, d1: bool = False) -> Result:
    """The oracle on one field.  ``threads`` > 1 spreads the lower stars of
    the gradient step over host threads by z-slabs (same result); every
    other step is single-threaded.  ``d1`` adds the saddle-saddle pairs
    (Alg. 2-3, after D0 and D2)."""
    flags = (RUN_ORDER if order else 0) | (RUN_GRADIENT if gradient else 0) \
        | (RUN_DIAGRAMS if diagrams else 0) | (RUN_REDUCTION if reduction else 0) \
        | (RUN_D1 if d1 else 0)
    return Result(field, flags, threads)


def pair_extrema_saddles(t0, t1, rank) -> np.ndarray:
    """Alg. 1 on an abstract extremum graph: triplets (sigma_j, t0[j], t1[j]) in
    visiting order, extrema compared by ``rank`` (higher = younger, dies).
    Returns, per triplet, the extremum paired with it, or -1."""
    t0 = np.ascontiguousarray(t0, dtype=np.int64)
    t1 = np.ascontiguousarray(t1, dtype=np.int64)
    rank = np.ascontiguousarray(rank, dtype=np.int64)
    out = np.empty(len(t0), dtype=np.int64)
    _load().orc_pair_extrema_saddles(len(t0), t0.ctypes.data, t1.ctypes.data, len(rank),
                                     rank.ctypes.data, out.ctypes.data)
    return out


def lower_star_vertex(field: np.ndarray, v: int):
    """ProcessLowerStars of one vertex straight from the field (no global sort).
    Returns (pairs[k,3] as (tail_dim, tail_id, head_id), crit[m,2] as (dim, id))."""
    f = np.ascontiguousarray(field, dtype=np.float32)
    nz, ny, nx = f.shape
    pairs = np.empty((80, 3), dtype=np.int64)
    crit = np.empty((80, 2), dtype=np.int64)
    n_p = ctypes.c_int64()
    n_c = ctypes.c_int64()
    rc = _load().orc_lower_star_vertex(f.ctypes.data, nx, ny, nz, int(v), pairs.ctypes.data, 80,
                                       ctypes.byref(n_p), crit.ctypes.data, 80, ctypes.byref(n_c))
    if rc:
        raise OracleError("lower star capacity")
    return pairs[: n_p.value].copy(), crit[: n_c.value].copy()


def _local(name, field, sid, limit):
    f = np.ascontiguousarray(field, dtype=np.float32)
    nz, ny, nx = f.shape
    out = ctypes.c_int64(-3)
    rc = getattr(_load(), name)(f.ctypes.data, nx, ny, nz, int(sid), int(limit), ctypes.byref(out))
    if rc == -2:
        raise OracleError("no such simplex")
    return rc, int(out.value)


def d0_edge_local(field: np.ndarray, edge: int, limit: int = 1 << 62):
    """Elder rule at one edge, by growing the two sublevel components at its
    ends (Sec. 2.4): (1, dying minimum) if the edge kills a component, (0, -3)
    if its ends are already connected, (-1, -3) past `limit` vertices."""
    return _local("orc_d0_edge_local", field, edge, limit)


def d2_triangle_local(field: np.ndarray, tri: int, limit: int = 1 << 62):
    """Dual elder rule at one triangle on tetrahedra + the outside:
    (1, dying tetrahedron), (0, -3) or (-1, -3) as in d0_edge_local."""
    return _local("orc_d2_triangle_local", field, tri, limit)


# ---------------------------------------------------------------- 2D grids --
# selectors of orc2_copy (mirror the enum in dms_oracle2d.cpp)
ORDER2, CRIT2_0, CRIT2_1, CRIT2_2, GRAD_PAIRS2, D0_2, D1_2, D0_ESSENTIAL2, REDUCTION2 = range(9)


class Result2:
    """Everything the 2D oracle computed for one field [ny, nx]."""

    def __init__(self, field: np.ndarray, flags: int):
        f = np.ascontiguousarray(field, dtype=np.float32)
        if f.ndim != 2:
            raise ValueError("field must be 2D, indexed [y, x]")
        ny, nx = f.shape
        lib = _load()
        self._h = lib.orc2_run(f.ctypes.data, nx, ny, flags)
        st = lib.orc2_status(self._h)
        if st:
            lib.orc2_free(self._h)
            self._h = None
            raise OracleError(_STATUS.get(st, f"status {st}"))

    def get(self, what: int) -> np.ndarray:
        lib = _load()
        n = lib.orc2_count(self._h, what)
        if what in (D0_2, D1_2, D0_ESSENTIAL2):
            out = np.empty(n, dtype=PAIR_DTYPE)
        elif what == ORDER2:
            out = np.empty(n, dtype=np.uint32)
        else:
            out = np.empty(n, dtype=np.int64)
        if n:
            lib.orc2_copy(self._h, what, out.ctypes.data)
        if what in (GRAD_PAIRS2, REDUCTION2):
            out = out.reshape(-1, 3)
        return out

    @property
    def order(self):
        return self.get(ORDER2)

    def crit(self, d: int) -> np.ndarray:
        return self.get(CRIT2_0 + d)

    def __del__(self):
        if getattr(self, "_h", None) is not None:
            _load().orc2_free(self._h)
            self._h = None


def run2(field: np.ndarray, diagrams=True, reduction=False) -> Result2:
    """The 2D oracle on a field indexed [y, x]: order, gradient, critical
    simplices and (by default) the D0 / D1 pairs; the boundary-matrix
    reduction on request (small grids only)."""
    flags = 1 | 2 | (4 if diagrams else 0) | (8 if reduction else 0)
    return Result2(field, flags)
