"""Batched diagrams of many fields of uneven dims (dms_batch_diagrams).

``Batch`` owns every device buffer for one fixed list of field shapes, so a
call allocates nothing and synchronises nothing: it can be captured once in a
CUDA graph and replayed for each new batch of inputs.  ``autotune`` picks the
gradient variant -- tile shape and lanes per vertex -- for a list of shapes
by timing the compiled variants and keeps the winner in a small JSON cache.  ``per_field`` runs the same fields
one at a time through the single-field entry points (the comparison point for
the batched path).
"""
from __future__ import annotations

import ctypes
import hashlib
import json
import os

import numpy as np
import torch

from . import _lib
from .api import PAIR_BYTES, PAIR_DTYPE, DMSError, _check, _ptr, _stream, diagram


def _field_table(shapes):
    n = len(shapes)
    table = (_lib.dms_field_desc * n)()
    off = 0
    for i, (nz, ny, nx) in enumerate(shapes):
        table[i].offset = off
        table[i].nx, table[i].ny, table[i].nz, table[i].reserved = nx, ny, nz, 0
        off += nx * ny * nz
    return table, off


class Batch:
    """Buffers and launch of ``dms_batch_diagrams`` for a fixed list of shapes
    (each ``(nz, ny, nx)``).

    ``caps`` are the capacities of the four critical lists over the whole
    batch; by default they start from a bound that holds for white noise and
    grow (one host sync) when ``fit()`` finds them too small.
    """

    def __init__(self, shapes, device="cuda", tile_variant: int = 0, caps=None):
        self.lib = _lib.load()
        self.shapes = [tuple(int(v) for v in s) for s in shapes]
        if not self.shapes:
            raise ValueError("a batch needs at least one field")
        self.device = torch.device(device)
        self.nfields = len(self.shapes)
        self.table, self.total = _field_table(self.shapes)
        self.sizes = [nz * ny * nx for nz, ny, nx in self.shapes]
        self.offsets = np.concatenate([[0], np.cumsum(self.sizes)]).astype(np.int64)
        raw = bytes(memoryview(self.table).cast("B"))
        self.table_dev = torch.frombuffer(bytearray(raw), dtype=torch.uint8).to(self.device)
        self.tile_variant = int(tile_variant)
        if not 0 <= self.tile_variant < self.lib.dms_batch_tile_variants():
            raise ValueError("tile_variant out of range")
        dev = self.device
        self.f = torch.zeros(self.total, dtype=torch.float32, device=dev)
        self.order = torch.empty(self.total, dtype=torch.uint32, device=dev)
        self.desc = torch.empty(self.total, dtype=torch.uint8, device=dev)
        self.rec = torch.empty(self.total, dtype=torch.int64, device=dev)
        self.counts = torch.zeros(6, dtype=torch.int64, device=dev)
        self.pair_offsets = torch.zeros((2, self.nfields + 1), dtype=torch.int64, device=dev)
        self.essential = torch.zeros((self.nfields, PAIR_BYTES), dtype=torch.uint8, device=dev)
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)
        if caps is None:
            t = self.total
            caps = [t // 8 + 64, t // 4 + 64, t // 4 + 64, t // 8 + 64]
        self._size(caps)

    def _size(self, caps):
        self.caps = [int(c) for c in caps]
        self.cap_pairs = max(self.caps[0], self.caps[3], 1)
        dev = self.device
        self.d0 = torch.empty((self.cap_pairs, PAIR_BYTES), dtype=torch.uint8, device=dev)
        self.d2 = torch.empty((self.cap_pairs, PAIR_BYTES), dtype=torch.uint8, device=dev)
        self._caps_arr = (ctypes.c_int64 * 4)(*self.caps)
        nbytes = self.lib.dms_batch_workspace_size(ctypes.byref(self.table), self.nfields,
                                                   self._caps_arr, self.cap_pairs)
        if nbytes == 0:
            raise ValueError("invalid batch (dims, total size or capacities)")
        self.ws = torch.empty(int(nbytes), dtype=torch.uint8, device=dev)

    # ------------------------------------------------------------ inputs --
    def field_view(self, i: int) -> torch.Tensor:
        """Field i of the flat input buffer, shaped [nz, ny, nx]."""
        a, b = int(self.offsets[i]), int(self.offsets[i + 1])
        return self.f[a:b].view(self.shapes[i])

    def set_fields(self, fields):
        for i, x in enumerate(fields):
            self.field_view(i).copy_(torch.as_tensor(x).reshape(self.shapes[i]), non_blocking=True)

    # ------------------------------------------------------------ launch --
    def launch(self, stream=None):
        """Enqueue the whole batch on the current (or given) stream; no sync."""
        s = stream.cuda_stream if stream is not None else _stream(self.device)
        self.status.zero_()
        _check(self.lib.dms_batch_diagrams(
            _ptr(self.f), ctypes.byref(self.table), _ptr(self.table_dev), self.nfields,
            self.tile_variant, _ptr(self.order), _ptr(self.desc), _ptr(self.rec), self._caps_arr,
            self.cap_pairs, _ptr(self.d0), _ptr(self.d2), _ptr(self.pair_offsets),
            _ptr(self.essential), _ptr(self.counts), _ptr(self.ws), self.ws.numel(),
            _ptr(self.status), s), "dms_batch_diagrams")

    def status_code(self) -> int:
        v = int(self.status.item())
        for c in range(1, 9):
            if v & (1 << c):
                return c
        return 0

    def fit(self, max_tries: int = 4):
        """Launch, and grow the capacities until every list fits (syncs)."""
        for _ in range(max_tries):
            self.launch()
            code = self.status_code()
            if code == 0:
                return self
            if code != 4:  # DMS_ERR_CAPACITY
                raise DMSError(code, "dms_batch_diagrams")
            n = [int(x) for x in self.counts.cpu()]
            self._size([max(c, int(k * 1.25) + 64) for c, k in zip(self.caps, n[:4])])
        raise DMSError(4, "dms_batch_diagrams")

    def check(self):
        code = self.status_code()
        if code:
            raise DMSError(code, "dms_batch_diagrams")

    # ------------------------------------------------------------- graph --
    def capture(self):
        """Capture one launch in a CUDA graph (after a launch outside it)."""
        self.fit()
        torch.cuda.synchronize(self.device)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.launch()
        return self.graph

    def replay(self):
        self.graph.replay()

    # ----------------------------------------------------------- results --
    def results(self):
        """Per field: (D0 pairs, D2 pairs, essential pair) as numpy
        structured arrays (PAIR_DTYPE), ids local to the field."""
        self.check()
        offs = self.pair_offsets.cpu().numpy()
        d0 = self.d0[: int(offs[0, -1])].cpu().numpy().view(PAIR_DTYPE).reshape(-1)
        d2 = self.d2[: int(offs[1, -1])].cpu().numpy().view(PAIR_DTYPE).reshape(-1)
        ess = self.essential.cpu().numpy().view(PAIR_DTYPE).reshape(-1)
        return [(d0[offs[0, i]:offs[0, i + 1]], d2[offs[1, i]:offs[1, i + 1]], ess[i:i + 1])
                for i in range(self.nfields)]


def per_field(fields):
    """The comparison point: each field through the single-field path."""
    out = []
    for x in fields:
        r = diagram(x)
        out.append((r.diagrams.numpy("d0"), r.diagrams.numpy("d2"),
                    r.diagrams.numpy("d0_essential")))
    return out


# ---------------------------------------------------------------- tuning --

def _cache_path():
    return os.environ.get("DMS_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "dms_gb300",
                                       "autotune.json"))


def _key(shapes, device):
    h = hashlib.sha1(json.dumps(sorted(shapes)).encode()).hexdigest()[:16]
    return f"{torch.cuda.get_device_name(device)}|{len(shapes)}|{h}"


def variant_name(v: int) -> str:
    """The gradient variant v: anchors per CTA tile and lanes per vertex."""
    return f"32x{(24, 16, 32)[v % 3]}, {1 + v // 3} lane(s)/vertex"


def autotune(shapes, device="cuda", fields=None, reps: int = 3, use_cache: bool = True):
    """Best gradient variant (tile shape x lanes per vertex) for these shapes,
    timed on the device with CUDA events over graph replays of the whole
    batch; cached by device name and shape list.  The times of the last
    call (ms per variant) are left in ``autotune.last``."""
    shapes = [tuple(int(v) for v in s) for s in shapes]
    key = _key(shapes, device)
    path = _cache_path()
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            cache = json.load(open(path))
        except (OSError, ValueError):
            cache = {}
        if key in cache:
            autotune.last = dict(cache[key])
            return int(cache[key]["variant"])
    times = []
    nvar = _lib.load().dms_batch_tile_variants()
    for v in range(nvar):
        b = Batch(shapes, device, tile_variant=v)
        if fields is not None:
            b.set_fields(fields)
        b.capture()
        b.replay()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            b.replay()
        e1.record()
        torch.cuda.synchronize(device)
        b.check()
        times.append(e0.elapsed_time(e1) / reps)
        del b
    best = int(np.argmin(times))
    autotune.last = {"variant": best, "ms": times}
    if use_cache:
        cache[key] = {"variant": best, "ms": times}
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            with open(path, "w") as fh:
                json.dump(cache, fh, indent=1)
        except OSError:
            pass
    return best


autotune.last = None
