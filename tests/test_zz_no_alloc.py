"""dms_critical_noalloc against dms_critical, through the C ABI.

The no-alloc entry point serves callers that cannot allocate device memory
(allocator-free regions of a host framework, plug-ins that only receive their
buffers, loops that must not call cudaMalloc): its scratch is a static array
in the library.  Its output must equal the workspace-based entry point's,
exactly (integer ids), on two calls in a row -- the second call runs on the
scratch the first one left behind.  This file sorts last so a failure here
does not hide any other test.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2505_21266_gb300 as dms
from paper_2505_21266_gb300 import _lib, fields


def _call_noalloc(lib, g, caps):
    dev = g.desc.device
    lists = [torch.full((max(int(c), 1),), -7, dtype=torch.int64, device=dev) for c in caps]
    counts = torch.full((4,), -1, dtype=torch.int64, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    nz, ny, nx = g.desc.shape
    cap = (ctypes.c_int64 * 4)(*[int(c) for c in caps])
    rc = lib.dms_critical_noalloc(ctypes.c_void_p(g.desc.data_ptr()), ctypes.c_void_p(g.rec.data_ptr()),
                                  _lib.dms_dims(nx, ny, nz),
                                  *[ctypes.c_void_p(t.data_ptr()) for t in lists], cap,
                                  ctypes.c_void_p(counts.data_ptr()), ctypes.c_void_p(st.data_ptr()),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert rc == 0, _lib.status_name(rc)
    assert int(st.item()) == 0
    n = [int(x) for x in counts.cpu()]
    return [lists[k][: n[k]].cpu().numpy() for k in range(4)], n


@pytest.mark.parametrize("shape", [(37, 41, 43), (64, 64, 64)])
def test_noalloc_matches_critical_twice(shape):
    lib = _lib.load()
    f = torch.from_numpy(fields.uniform01(shape, 5).numpy()).cuda()
    g = dms.gradient(dms.order(f))
    ref = dms.critical(g)
    ref = [r.cpu().numpy() for r in ref]
    caps = [len(r) for r in ref]
    for _ in range(2):
        got, n = _call_noalloc(lib, g, caps)
        assert n == caps
        for k in range(4):
            assert np.array_equal(got[k], ref[k])


def test_noalloc_second_field_after_first():
    """A different, smaller field right after a larger one: the scratch left
    by the previous call must not leak into the result."""
    lib = _lib.load()
    for shape, seed in (((50, 50, 50), 1), ((9, 30, 17), 2)):
        f = torch.from_numpy(fields.quantized_noise(shape, 16, seed).numpy()).cuda()
        g = dms.gradient(dms.order(f))
        ref = [r.cpu().numpy() for r in dms.critical(g)]
        got, n = _call_noalloc(lib, g, [len(r) for r in ref])
        for k in range(4):
            assert np.array_equal(got[k], ref[k])


def test_noalloc_rejects_too_large_grid():
    lib = _lib.load()
    assert lib.dms_critical_noalloc_max_vertices() == 1 << 30
    cap = (ctypes.c_int64 * 4)(0, 0, 0, 0)
    dummy = torch.zeros(16, dtype=torch.int64, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    rc = lib.dms_critical_noalloc(p, p, _lib.dms_dims(2048, 1024, 1024), None, None, None, None,
                                  cap, p, p, None)
    assert rc == 9  # DMS_ERR_TOO_LARGE, before any launch
