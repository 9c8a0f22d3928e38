"""The C-ABI calls accept caller buffers at any address their element type
allows: dms_critical on gradient records and bytes that do not start on a
16-byte boundary (the element-by-element staging path) must give the same
lists as on the library's own aligned buffers."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2505_21266_gb300 as dms
from paper_2505_21266_gb300 import _lib, fields


def _critical_at(lib, desc, rec, dims, caps):
    dev = desc.device
    lists = [torch.full((max(int(c), 1),), -7, dtype=torch.int64, device=dev) for c in caps]
    counts = torch.full((4,), -1, dtype=torch.int64, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    cap = (ctypes.c_int64 * 4)(*[int(c) for c in caps])
    ws = torch.empty(max(int(lib.dms_critical_workspace_size(dims)), 256), dtype=torch.uint8,
                     device=dev)
    rc = lib.dms_critical(ctypes.c_void_p(desc.data_ptr()), ctypes.c_void_p(rec.data_ptr()), dims,
                          *[ctypes.c_void_p(t.data_ptr()) for t in lists], cap,
                          ctypes.c_void_p(counts.data_ptr()), ctypes.c_void_p(ws.data_ptr()),
                          ws.numel(), ctypes.c_void_p(st.data_ptr()),
                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert rc == 0, _lib.status_name(rc)
    assert int(st.item()) == 0
    n = [int(x) for x in counts.cpu()]
    return [lists[k][: n[k]].cpu().numpy() for k in range(4)]


@pytest.mark.parametrize("shape", [(40, 41, 43), (64, 64, 70)])
def test_critical_on_unaligned_buffers(shape):
    lib = _lib.load()
    f = torch.from_numpy(fields.uniform01(shape, 11).numpy()).cuda()
    g = dms.gradient(dms.order(f))
    ref = [r.cpu().numpy() for r in dms.critical(g)]
    caps = [len(r) for r in ref]
    nz, ny, nx = shape
    n = nx * ny * nz
    # the same bytes one byte (desc) and one record (rec) past a 16-byte boundary
    dbuf = torch.zeros(n + 16, dtype=torch.uint8, device="cuda")
    rbuf = torch.zeros(n + 2, dtype=torch.int64, device="cuda")
    desc = dbuf[1:1 + n]
    rec = rbuf[1:1 + n]
    desc.copy_(g.desc.reshape(-1))
    rec.copy_(g.rec.reshape(-1).view(torch.int64))
    assert desc.data_ptr() % 16 != 0 and rec.data_ptr() % 16 != 0
    got = _critical_at(lib, desc, rec, _lib.dms_dims(nx, ny, nz), caps)
    for k in range(4):
        assert np.array_equal(got[k], ref[k]), k
