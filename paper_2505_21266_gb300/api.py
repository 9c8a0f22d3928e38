"""Python front end of the DMS hot path: argument marshalling around the C ABI.

Tensors are torch CUDA tensors (PyTorch provides device memory and streams);
every computation runs in ``libdms_gb300.so``.  Fields are indexed
``field[z, y, x]`` (x fastest, the vertex offset v = x + nx*(y + ny*z)).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib

PAIR_DTYPE = np.dtype([("birth_id", "<i8"), ("death_id", "<i8"), ("birth", "<f4"),
                       ("death", "<f4"), ("birth_vtx", "<u4"), ("death_vtx", "<u4")])
PAIR_BYTES = 32
CRITICAL = 7  # record code of a critical edge / tetrahedron


class DMSError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = int(code)
        super().__init__(f"{where}: {_lib.status_name(code)}")


def _check(rc: int, where: str):
    if rc != 0:
        raise DMSError(rc, where)


def _device_status_check(st: torch.Tensor, where: str):
    v = int(st.item())
    if v:
        codes = [c for c in range(1, 9) if v & (1 << c)]
        raise DMSError(codes[0], where)


def dims_of(field: torch.Tensor) -> _lib.dms_dims:
    if field.dim() != 3:
        raise ValueError("field must be a 3D tensor indexed [z, y, x]")
    nz, ny, nx = field.shape
    return _lib.dms_dims(nx, ny, nz)


def _require_cuda(t: torch.Tensor, name: str, dtype=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (the DMS library has no CPU path)")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def _require_gradient(g, rec_dtype):
    """A gradient's arrays: on the device, contiguous, of one shape."""
    _require_cuda(g.desc, "gradient desc", torch.uint8)
    _require_cuda(g.rec, "gradient rec", rec_dtype)
    if g.rec.shape != g.desc.shape or g.rec.device != g.desc.device:
        raise ValueError("gradient rec and desc must have the same shape and device")


def _stream(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _to_host(t: torch.Tensor) -> torch.Tensor:
    """A host copy of t; device tensors land in page-locked memory (the copy
    runs at the link's rate, and torch's host allocator reuses the buffers)."""
    if not t.is_cuda:
        return t
    h = torch.empty(t.shape, dtype=t.dtype, pin_memory=True)
    h.copy_(t)
    return h


def _ws(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


# ------------------------------------------------------------------- (i) --

def order(field: torch.Tensor, status: torch.Tensor | None = None, check: bool = True):
    """Global vertex order (Sec. 2.1, Sec. 3): uint32 tensor shaped like field."""
    _require_cuda(field, "field", torch.float32)
    lib = _lib.load()
    d = dims_of(field)
    out = torch.empty(field.shape, dtype=torch.uint32, device=field.device)
    ws = _ws(lib.dms_order_workspace_size(d), field.device)
    st = status if status is not None else torch.zeros(1, dtype=torch.int32, device=field.device)
    _check(lib.dms_order(_ptr(field), d, _ptr(out), _ptr(ws), ws.numel(), _ptr(st),
                         _stream(field.device)), "dms_order")
    if check and status is None:
        _device_status_check(st, "dms_order")
    return out


# ------------------------------------------------------------------ (ii) --

@dataclass
class Gradient:
    desc: torch.Tensor    # uint8 [nz, ny, nx]
    rec: torch.Tensor     # int64 [nz, ny, nx] (bit pattern of the uint64 records)
    counts: torch.Tensor  # int64 [4] critical simplices per dimension


def gradient(order_t: torch.Tensor) -> Gradient:
    """Robins et al.'s lower-star discrete gradient (Sec. 2.3)."""
    _require_cuda(order_t, "order", torch.uint32)
    lib = _lib.load()
    d = dims_of(order_t)
    desc = torch.empty(order_t.shape, dtype=torch.uint8, device=order_t.device)
    rec = torch.empty(order_t.shape, dtype=torch.int64, device=order_t.device)
    counts = torch.empty(4, dtype=torch.int64, device=order_t.device)
    _check(lib.dms_gradient(_ptr(order_t), d, _ptr(desc), _ptr(rec), _ptr(counts),
                            _stream(order_t.device)), "dms_gradient")
    return Gradient(desc, rec, counts)


# ----------------------------------------------------------------- (iii) --

def critical(g: Gradient, caps=None, status: torch.Tensor | None = None):
    """Critical simplices per dimension, each list sorted by id (int64).
    Without ``caps`` the capacities are read from ``g.counts`` (one sync)."""
    _require_gradient(g, torch.int64)
    lib = _lib.load()
    dev = g.desc.device
    d = dims_of(g.desc)
    if caps is None:
        caps = [int(x) for x in g.counts.cpu()]
        if caps[0] < 0:  # a TMA copy of the order field did not land: invalid gradient
            raise DMSError(7, "dms_gradient")  # DMS_ERR_TIMEOUT
    lists = [torch.empty(max(int(c), 1), dtype=torch.int64, device=dev) for c in caps]
    cap_arr = (ctypes.c_int64 * 4)(*[int(c) for c in caps])
    counts = torch.empty(4, dtype=torch.int64, device=dev)
    ws = _ws(lib.dms_critical_workspace_size(d), dev)
    st = status if status is not None else torch.zeros(1, dtype=torch.int32, device=dev)
    _check(lib.dms_critical(_ptr(g.desc), _ptr(g.rec), d, *[_ptr(t) for t in lists], cap_arr,
                            _ptr(counts), _ptr(ws), ws.numel(), _ptr(st), _stream(dev)),
           "dms_critical")
    if status is None:
        _device_status_check(st, "dms_critical")
        n = [int(x) for x in counts.cpu()]
        return [lists[k][: n[k]] for k in range(4)]
    return lists, counts


# ------------------------------------------------------------------ (iv) --

@dataclass
class Diagrams:
    d0: torch.Tensor           # uint8 [n0, 32] pair records (see PAIR_DTYPE)
    d2: torch.Tensor           # uint8 [n2, 32]
    d0_essential: torch.Tensor  # uint8 [1, 32]

    def numpy(self, which: str) -> np.ndarray:
        return _to_host(getattr(self, which)).numpy().view(PAIR_DTYPE).reshape(-1)


def diagram_d0d2(field: torch.Tensor, order_t: torch.Tensor, g: Gradient, crit,
                 status: torch.Tensor | None = None, pairing: str = "rounds") -> Diagrams:
    """D0 and D2 pairs (Sec. 2.5, Alg. 1 and its dual; Sec. 4).  ``pairing``
    picks the parallel form of Alg. 1: "rounds" (spanning forest, then exact
    rounds; the default) or "selfcorrecting" (the paper's self-correcting
    pairing, Alg. 4, as a fixpoint); both give Alg. 1's pairs."""
    if pairing not in ("rounds", "selfcorrecting"):
        raise ValueError("pairing is 'rounds' or 'selfcorrecting'")
    _require_cuda(field, "field", torch.float32)
    lib = _lib.load()
    dev = field.device
    d = dims_of(field)
    nc = [int(c.numel()) for c in crit]
    ncarr = (ctypes.c_int64 * 4)(*nc)
    cap0, cap2 = max(nc[0] - 1, 0), nc[3]
    d0 = torch.empty((max(cap0, 1), PAIR_BYTES), dtype=torch.uint8, device=dev)
    d2 = torch.empty((max(cap2, 1), PAIR_BYTES), dtype=torch.uint8, device=dev)
    ess = torch.zeros((1, PAIR_BYTES), dtype=torch.uint8, device=dev)
    n_out = torch.zeros(2, dtype=torch.int64, device=dev)
    ws = _ws(lib.dms_diagram_workspace_size(d, ncarr), dev)
    st = status if status is not None else torch.zeros(1, dtype=torch.int32, device=dev)
    crit_p = [_ptr(c) if c.numel() else None for c in crit]
    fn = lib.dms_diagram_d0d2 if pairing == "rounds" else lib.dms_diagram_d0d2_selfcorrecting
    _check(fn(_ptr(field), _ptr(order_t), _ptr(g.desc), _ptr(g.rec), d, *crit_p, ncarr, _ptr(d0),
              cap0, _ptr(d2), cap2, _ptr(ess), _ptr(n_out), _ptr(ws), ws.numel(), _ptr(st),
              _stream(dev)), "dms_diagram_d0d2")
    if status is None:
        _device_status_check(st, "dms_diagram_d0d2")
    n = [int(x) for x in n_out.cpu()]
    return Diagrams(d0[: n[0]], d2[: n[1]], ess)


# boundary-pool entries per critical triangle that the last D1 call needed
# (the library's default is 256); later calls start from it
_d1_pool_ratio = [256]


def diagram_d1(field: torch.Tensor, order_t: torch.Tensor, g: Gradient, crit, dg: Diagrams,
               pool_entries: int = 0, max_tries: int = 4) -> torch.Tensor:
    """D1 pairs (birth = critical edge, death = critical triangle) of a 3D
    field after its D0 / D2 pairs (Sec. 2.5, Alg. 2 and Alg. 3), as pair
    records [n1, 32] in increasing triangle-id order.  The boundary pool
    grows (the call is repeated) when a boundary outgrows it, and the size
    that worked is where the next call starts."""
    _require_cuda(field, "field", torch.float32)
    lib = _lib.load()
    dev = field.device
    d = dims_of(field)
    nc = [int(c.numel()) for c in crit]
    ncarr = (ctypes.c_int64 * 4)(*nc)
    n_d0, n_d2 = int(dg.d0.shape[0]), int(dg.d2.shape[0])
    cap1 = max(nc[2] - n_d2, 0)
    out = torch.empty((max(cap1, 1), PAIR_BYTES), dtype=torch.uint8, device=dev)
    n_out = torch.zeros(1, dtype=torch.int64, device=dev)
    ratio = _d1_pool_ratio[0]
    pool = int(pool_entries) if pool_entries else ratio * max(nc[2], 1) + 65536
    if not pool_entries:
        # a repeated call starts from scratch, so the first one gets as much
        # of the free memory as the ratio asks for (16-byte entries, a fifth
        # of the free memory left for the rest of the workspace)
        free = torch.cuda.mem_get_info(dev)[0]
        pool = max(min(pool, int(free * 0.8) // 16), 16 * max(nc[2], 1) + 65536)
    for _ in range(max_tries):
        ws = _ws(lib.dms_diagram_d1_workspace_size(d, ncarr, pool), dev)
        st = torch.zeros(1, dtype=torch.int32, device=dev)
        _check(lib.dms_diagram_d1(_ptr(field), _ptr(order_t), _ptr(g.rec), d,
                                  _ptr(crit[1]) if nc[1] else None,
                                  _ptr(crit[2]) if nc[2] else None, ncarr,
                                  _ptr(dg.d0) if n_d0 else None, n_d0,
                                  _ptr(dg.d2) if n_d2 else None, n_d2, _ptr(out), cap1,
                                  _ptr(n_out), pool, _ptr(ws), ws.numel(), _ptr(st),
                                  _stream(dev)), "dms_diagram_d1")
        v = int(st.item())
        if v == (1 << 4):  # the pool only: retry with four times as much
            pool *= 4
            ratio *= 4
            continue
        _device_status_check(st, "dms_diagram_d1")
        if not pool_entries:
            _d1_pool_ratio[0] = ratio
        return out[: int(n_out.item())]
    raise DMSError(4, "dms_diagram_d1")


@dataclass
class Result:
    order: torch.Tensor
    grad: Gradient
    crit: list
    diagrams: Diagrams


def diagram(field: torch.Tensor, pairing: str = "rounds") -> Result:
    """The whole hot path: order -> gradient -> critical simplices -> D0/D2."""
    o = order(field)
    g = gradient(o)
    c = critical(g)
    dg = diagram_d0d2(field, o, g, c, pairing=pairing)
    return Result(o, g, c, dg)


def diagram_from_host(field_host, device="cuda"):
    """End-to-end call for data that lives in host memory: copies the field to
    the device, runs the whole path, and returns the D0 / D2 pairs and the
    essential class as numpy structured arrays (PAIR_DTYPE)."""
    if not isinstance(field_host, torch.Tensor):
        field_host = torch.from_numpy(np.ascontiguousarray(field_host, dtype=np.float32))
    f = field_host.to(device, non_blocking=True)
    res = diagram(f)
    return (res.diagrams.numpy("d0"), res.diagrams.numpy("d2"),
            res.diagrams.numpy("d0_essential"))


def diagrams_from_host(fields_host, device="cuda"):
    """End-to-end for a sequence of fields in host memory (page-locked for
    the copies to overlap): yields, per field, its D0 / D2 pairs and
    essential class as numpy structured arrays, like diagram_from_host.
    The host-to-device copy of the next field runs on a separate stream
    while the current field goes through the path, into the second of two
    device buffers.  A field's pairs come back to page-locked host memory on
    a third stream once the next field's order and gradient kernels are
    queued: the path's small reads of counts go through the same
    device-to-host copy engine, and behind a copy of the pair lists they
    would wait for all of it, while the gradient kernel reads nothing on the
    host.  So a field's arrays are yielded after the next field's path."""
    dev = torch.device(device)
    compute = torch.cuda.current_stream(dev)
    copier = torch.cuda.Stream(dev)
    drain = torch.cuda.Stream(dev)
    bufs, ready = [None, None], [None, None]

    def enqueue(i, x):
        if not isinstance(x, torch.Tensor):
            x = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32))
        if bufs[i] is None or bufs[i].shape != x.shape:
            bufs[i] = torch.empty(x.shape, dtype=torch.float32, device=dev)
        if bufs[1 - i] is None:  # the other buffer too, at the first field
            bufs[1 - i] = torch.empty(x.shape, dtype=torch.float32, device=dev)
        copier.wait_stream(compute)  # the buffer's last reader is done
        with torch.cuda.stream(copier):
            bufs[i].copy_(x, non_blocking=True)
            ready[i] = torch.cuda.Event()
            ready[i].record(copier)

    def start_drain(dg, end):
        """A field's pair lists to page-locked host memory on `drain`, after
        the event `end` that closes the field's path."""
        drain.wait_event(end)
        outs = []
        with torch.cuda.stream(drain):
            for t in (dg.d0, dg.d2, dg.d0_essential):
                h = torch.empty(t.shape, dtype=t.dtype, pin_memory=True)
                h.copy_(t, non_blocking=True)
                t.record_stream(drain)  # the device list outlives the copy
                outs.append(h)
            done = torch.cuda.Event()
            done.record(drain)
        return outs, done

    def finish(p):
        outs, done = p
        done.synchronize()
        return tuple(h.numpy().view(PAIR_DTYPE).reshape(-1) for h in outs)

    it = iter(fields_host)
    nxt = next(it, None)
    if nxt is None:
        return
    cur = 0
    enqueue(cur, nxt)
    prev = None  # the last field's pair lists and the event after its path
    while True:
        compute.wait_event(ready[cur])
        nxt = next(it, None)
        if nxt is not None:
            enqueue(1 - cur, nxt)  # overlaps the path below
        f = bufs[cur]
        st = torch.zeros(1, dtype=torch.int32, device=dev)
        o = order(f, status=st)
        g = gradient(o)
        p = start_drain(*prev) if prev is not None else None
        prev = None
        _device_status_check(st, "dms_order")
        dg = diagram_d0d2(f, o, g, critical(g))
        end = torch.cuda.Event()
        end.record(compute)
        prev = (dg, end)
        del o, g, dg
        if p is not None:
            yield finish(p)  # the previous field; its copy ran behind this gradient
        if nxt is None:
            break
        cur = 1 - cur
    yield finish(start_drain(*prev))


# ------------------------------------------------------------------ diff --

def pair_values(pairs: torch.Tensor) -> torch.Tensor:
    """(birth, death) float32 values [n, 2] of pair records [n, 32]."""
    return pairs.view(torch.float32).reshape(-1, PAIR_BYTES // 4)[:, 4:6]


def backward(pairs: torch.Tensor, g: torch.Tensor, grad: torch.Tensor,
             status: torch.Tensor | None = None):
    """grad[carrier] += dL/d(value) for every pair (dms_backward): pairs
    [n, 32] pair records, g [n, 2] (dL/dbirth, dL/ddeath), grad the field's
    gradient (float32), all on the device."""
    _require_cuda(pairs, "pairs", torch.uint8)
    _require_cuda(grad, "grad", torch.float32)
    if pairs.dim() != 2 or pairs.shape[1] != PAIR_BYTES:
        raise ValueError(f"pairs must be [n, {PAIR_BYTES}] pair records")
    lib = _lib.load()
    g = g.to(torch.float32).contiguous()
    _require_cuda(g, "g", torch.float32)
    n = int(pairs.shape[0])
    if g.numel() != 2 * n:
        raise ValueError("g must hold (dL/dbirth, dL/ddeath) for every pair")
    if n == 0:
        return grad
    st = status if status is not None else torch.zeros(1, dtype=torch.int32, device=grad.device)
    _check(lib.dms_backward(_ptr(pairs), n, _ptr(g), dims_of(grad), _ptr(grad), _ptr(st),
                            _stream(grad.device)), "dms_backward")
    if status is None:
        _device_status_check(st, "dms_backward")
    return grad


class DiagramFn(torch.autograd.Function):
    """Differentiable D0/D2 diagrams: forward returns the (birth, death) values
    of the D0 and D2 pairs; backward scatter-adds the incoming gradients onto
    the carrier vertices with the dms_backward kernel."""

    @staticmethod
    def forward(ctx, field):
        res = diagram(field.detach().contiguous())
        d0, d2 = res.diagrams.d0, res.diagrams.d2
        ctx.save_for_backward(d0, d2)
        ctx.field_shape = field.shape
        return pair_values(d0).clone(), pair_values(d2).clone()

    @staticmethod
    def backward(ctx, g0, g2):
        d0, d2 = ctx.saved_tensors
        grad = torch.zeros(ctx.field_shape, dtype=torch.float32, device=d0.device)
        if g0 is not None and d0.shape[0]:
            backward(d0, g0, grad)
        if g2 is not None and d2.shape[0]:
            backward(d2, g2, grad)
        return grad


def diagram_values(field: torch.Tensor):
    """Autograd entry point: (D0 values [n0, 2], D2 values [n2, 2])."""
    return DiagramFn.apply(field)


def topological_loss(field: torch.Tensor, threshold: float = 0.05) -> torch.Tensor:
    """Sum over the D0 and D2 pairs with persistence below `threshold` of
    (death - birth)^2 -- a topological simplification loss."""
    v0, v2 = diagram_values(field)
    v = torch.cat([v0, v2])
    pers = v[:, 1] - v[:, 0]
    keep = pers < threshold
    return (pers[keep] ** 2).sum()


# -------------------------------------------------------------------- 2D --

def dims2_of(field: torch.Tensor):
    if field.dim() != 2:
        raise ValueError("a 2D field is a 2D tensor indexed [y, x]")
    ny, nx = field.shape
    return int(nx), int(ny)


def order2d(field: torch.Tensor, status: torch.Tensor | None = None, check: bool = True):
    """Global vertex order of a 2D field (Sec. 2.1): uint32, shaped like field."""
    _require_cuda(field, "field", torch.float32)
    lib = _lib.load()
    nx, ny = dims2_of(field)
    out = torch.empty(field.shape, dtype=torch.uint32, device=field.device)
    ws = _ws(lib.dms2_order_workspace_size(nx, ny), field.device)
    st = status if status is not None else torch.zeros(1, dtype=torch.int32, device=field.device)
    _check(lib.dms2_order(_ptr(field), nx, ny, _ptr(out), _ptr(ws), ws.numel(), _ptr(st),
                          _stream(field.device)), "dms2_order")
    if check and status is None:
        _device_status_check(st, "dms2_order")
    return out


@dataclass
class Gradient2d:
    desc: torch.Tensor  # uint8 [ny, nx]
    rec: torch.Tensor   # int16 [ny, nx] (bit pattern of the uint16 records)


def gradient2d(order_t: torch.Tensor) -> Gradient2d:
    """ProcessLowerStars on every vertex of a 2D grid (Sec. 2.3)."""
    _require_cuda(order_t, "order", torch.uint32)
    lib = _lib.load()
    nx, ny = dims2_of(order_t)
    desc = torch.empty(order_t.shape, dtype=torch.uint8, device=order_t.device)
    rec = torch.empty(order_t.shape, dtype=torch.int16, device=order_t.device)
    _check(lib.dms2_gradient(_ptr(order_t), nx, ny, _ptr(desc), _ptr(rec),
                             _stream(order_t.device)), "dms2_gradient")
    return Gradient2d(desc, rec)


def critical2d(g: Gradient2d, caps=None):
    """Critical vertices, edges and triangles of a 2D gradient, sorted by id.
    Without caps, a first call sizes the lists (one sync)."""
    _require_gradient(g, torch.int16)
    lib = _lib.load()
    dev = g.desc.device
    nx, ny = dims2_of(g.desc)
    ws = _ws(lib.dms2_critical_workspace_size(nx, ny), dev)
    counts = torch.empty(3, dtype=torch.int64, device=dev)

    def call(cap):
        lists = [torch.empty(max(int(c), 1), dtype=torch.int64, device=dev) for c in cap]
        st = torch.zeros(1, dtype=torch.int32, device=dev)
        cap_arr = (ctypes.c_int64 * 3)(*[int(c) for c in cap])
        _check(lib.dms2_critical(_ptr(g.desc), _ptr(g.rec), nx, ny, *[_ptr(t) for t in lists],
                                 cap_arr, _ptr(counts), _ptr(ws), ws.numel(), _ptr(st),
                                 _stream(dev)), "dms2_critical")
        return lists, st

    if caps is None:
        call([0, 0, 0])
        caps = [int(x) for x in counts.cpu()]
    lists, st = call(caps)
    _device_status_check(st, "dms2_critical")
    n = [int(x) for x in counts.cpu()]
    return [lists[k][: n[k]] for k in range(3)]


@dataclass
class Diagrams2d:
    d0: torch.Tensor            # uint8 [n0, 32] pair records (PAIR_DTYPE)
    d1: torch.Tensor            # uint8 [n1, 32]
    d0_essential: torch.Tensor  # uint8 [1, 32]

    def numpy(self, which: str) -> np.ndarray:
        return _to_host(getattr(self, which)).numpy().view(PAIR_DTYPE).reshape(-1)


def diagram_d0d1(field: torch.Tensor, order_t: torch.Tensor, g: Gradient2d, crit) -> Diagrams2d:
    """D0 and D1 pairs of a 2D field (Alg. 1 and its dual)."""
    _require_cuda(field, "field", torch.float32)
    lib = _lib.load()
    dev = field.device
    nx, ny = dims2_of(field)
    nc = [int(c.numel()) for c in crit]
    ncarr = (ctypes.c_int64 * 3)(*nc)
    cap0, cap1 = max(nc[0] - 1, 0), nc[2]
    d0 = torch.empty((max(cap0, 1), PAIR_BYTES), dtype=torch.uint8, device=dev)
    d1 = torch.empty((max(cap1, 1), PAIR_BYTES), dtype=torch.uint8, device=dev)
    ess = torch.zeros((1, PAIR_BYTES), dtype=torch.uint8, device=dev)
    n_out = torch.zeros(2, dtype=torch.int64, device=dev)
    ws = _ws(lib.dms2_diagram_workspace_size(nx, ny, ncarr), dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    crit_p = [_ptr(c) if c.numel() else None for c in crit]
    _check(lib.dms2_diagram_d0d1(_ptr(field), _ptr(order_t), _ptr(g.desc), _ptr(g.rec), nx, ny,
                                 *crit_p, ncarr, _ptr(d0), cap0, _ptr(d1), cap1, _ptr(ess),
                                 _ptr(n_out), _ptr(ws), ws.numel(), _ptr(st), _stream(dev)),
           "dms2_diagram_d0d1")
    _device_status_check(st, "dms2_diagram_d0d1")
    n = [int(x) for x in n_out.cpu()]
    return Diagrams2d(d0[: n[0]], d1[: n[1]], ess)


@dataclass
class Result2d:
    order: torch.Tensor
    grad: Gradient2d
    crit: list
    diagrams: Diagrams2d


def diagram2d(field: torch.Tensor) -> Result2d:
    """The whole path on a 2D field [y, x]: order, gradient, critical
    simplices, D0 and D1 (the full diagram of a 2D field)."""
    o = order2d(field)
    g = gradient2d(o)
    c = critical2d(g)
    return Result2d(o, g, c, diagram_d0d1(field, o, g, c))
