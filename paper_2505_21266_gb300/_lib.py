"""ctypes binding of ``libdms_gb300.so`` (the C ABI of ``include/dms.h``).

Argument marshalling only: every step of the path runs in the CUDA library.
Loading fails loudly when the library is missing -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

_lib = None


class dms_dims(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32)]


class dms_field_desc(ctypes.Structure):
    _fields_ = [("offset", ctypes.c_int64), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("nz", ctypes.c_int32), ("reserved", ctypes.c_int32)]


STATUS = {0: "DMS_OK", 1: "DMS_ERR_NULL", 2: "DMS_ERR_DIMS", 3: "DMS_ERR_NAN",
          4: "DMS_ERR_CAPACITY", 5: "DMS_ERR_WORKSPACE", 6: "DMS_ERR_CUDA",
          7: "DMS_ERR_TIMEOUT", 8: "DMS_ERR_ARG", 9: "DMS_ERR_TOO_LARGE"}

# (name, restype, argtypes) for every entry point declared in include/dms.h
_VP, _I64, _I32, _SZ = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_size_t
SIGNATURES = [
    ("dms_status_string", ctypes.c_char_p, [ctypes.c_int]),
    ("dms_launch_count", _I64, []),
    ("dms_num_vertices", _I64, [dms_dims]),
    ("dms_order_workspace_size", _SZ, [dms_dims]),
    ("dms_order", ctypes.c_int, [_VP, dms_dims, _VP, _VP, _SZ, _VP, _VP]),
    ("dms_gradient", ctypes.c_int, [_VP, dms_dims, _VP, _VP, _VP, _VP]),
    ("dms_critical_workspace_size", _SZ, [dms_dims]),
    ("dms_critical", ctypes.c_int,
     [_VP, _VP, dms_dims, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _SZ, _VP, _VP]),
    ("dms_critical_noalloc_max_vertices", _I64, []),
    ("dms_critical_noalloc", ctypes.c_int,
     [_VP, _VP, dms_dims, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    ("dms_backward", ctypes.c_int, [_VP, _I64, _VP, dms_dims, _VP, _VP, _VP]),
    ("dms_diagram_workspace_size", _SZ, [dms_dims, _VP]),
    ("dms_diagram_d0d2", ctypes.c_int,
     [_VP, _VP, _VP, _VP, dms_dims, _VP, _VP, _VP, _VP, _VP, _VP, _I64, _VP, _I64, _VP, _VP,
      _VP, _SZ, _VP, _VP]),
    ("dms_diagram_d0d2_selfcorrecting", ctypes.c_int,
     [_VP, _VP, _VP, _VP, dms_dims, _VP, _VP, _VP, _VP, _VP, _VP, _I64, _VP, _I64, _VP, _VP,
      _VP, _SZ, _VP, _VP]),
    ("dms_diagram_d1_workspace_size", _SZ, [dms_dims, _VP, _I64]),
    ("dms_diagram_d1", ctypes.c_int,
     [_VP, _VP, _VP, dms_dims, _VP, _VP, _VP, _VP, _I64, _VP, _I64, _VP, _I64, _VP, _I64, _VP,
      _SZ, _VP, _VP]),
    ("dms2_order_workspace_size", _SZ, [_I32, _I32]),
    ("dms2_order", ctypes.c_int, [_VP, _I32, _I32, _VP, _VP, _SZ, _VP, _VP]),
    ("dms2_gradient", ctypes.c_int, [_VP, _I32, _I32, _VP, _VP, _VP]),
    ("dms2_critical_workspace_size", _SZ, [_I32, _I32]),
    ("dms2_critical", ctypes.c_int,
     [_VP, _VP, _I32, _I32, _VP, _VP, _VP, _VP, _VP, _VP, _SZ, _VP, _VP]),
    ("dms2_diagram_workspace_size", _SZ, [_I32, _I32, _VP]),
    ("dms2_diagram_d0d1", ctypes.c_int,
     [_VP, _VP, _VP, _VP, _I32, _I32, _VP, _VP, _VP, _VP, _VP, _I64, _VP, _I64, _VP, _VP, _VP,
      _SZ, _VP, _VP]),
    ("dms_batch_tile_variants", _I32, []),
    ("dms_batch_max_rounds", _I32, []),
    ("dms_batch_workspace_size", _SZ, [_VP, _I32, _VP, _I64]),
    ("dms_batch_diagrams", ctypes.c_int,
     [_VP, _VP, _VP, _I32, _I32, _VP, _VP, _VP, _VP, _I64, _VP, _VP, _VP, _VP, _VP, _VP, _SZ,
      _VP, _VP]),
]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load the CUDA library (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing: run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def status_name(code: int) -> str:
    return STATUS.get(int(code), f"status {code}")
