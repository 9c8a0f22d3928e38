"""The Python binding has no CPU path: every entry point refuses host
tensors before anything runs, wrong dtypes and shapes are refused before a
kernel could index past a buffer, and a missing CUDA library is an error,
not a fallback.  Runs without a GPU."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2505_21266_gb300 as dms  # noqa: E402
from paper_2505_21266_gb300 import _lib, build  # noqa: E402


def _no_cpu(fn, *args):
    with pytest.raises(ValueError, match="CUDA tensor|no CPU path"):
        fn(*args)


def test_entry_points_refuse_host_tensors():
    f3 = torch.rand(4, 5, 6)
    f2 = torch.rand(5, 6)
    _no_cpu(dms.order, f3)
    _no_cpu(dms.gradient, torch.zeros(4, 5, 6, dtype=torch.uint32))
    _no_cpu(dms.diagram, f3)
    _no_cpu(dms.diagram_values, f3)
    _no_cpu(dms.order2d, f2)
    _no_cpu(dms.gradient2d, torch.zeros(5, 6, dtype=torch.uint32))
    _no_cpu(dms.diagram2d, f2)
    _no_cpu(dms.critical, dms.Gradient(torch.zeros(4, 5, 6, dtype=torch.uint8),
                                       torch.zeros(4, 5, 6, dtype=torch.int64),
                                       torch.zeros(4, dtype=torch.int64)))
    _no_cpu(dms.critical2d, dms.Gradient2d(torch.zeros(5, 6, dtype=torch.uint8),
                                           torch.zeros(5, 6, dtype=torch.int16)))
    rec = np.zeros(2, dtype=dms.PAIR_DTYPE)
    pairs = torch.from_numpy(rec.view(np.uint8).reshape(2, 32))
    _no_cpu(dms.backward, pairs, torch.zeros(2, 2), torch.zeros(2, 2, 2))


def test_library_missing_is_an_error(monkeypatch, tmp_path):
    monkeypatch.setattr(build, "LIB", str(tmp_path / "libdms_gb300.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        _lib.load(build_if_missing=False)


@pytest.mark.gpu
@pytest.mark.skipif(not torch.cuda.is_available(), reason="shape checks on device tensors")
def test_shapes_and_dtypes_are_checked_on_the_device():
    """Refused in the binding, before any launch."""
    dev = "cuda"
    pairs = torch.zeros(3, 32, dtype=torch.uint8, device=dev)
    grad = torch.zeros(2, 2, 2, device=dev)
    with pytest.raises(ValueError, match="every pair"):
        dms.backward(pairs, torch.zeros(2, 2, device=dev), grad)  # 2 value rows for 3 pairs
    with pytest.raises(ValueError, match="pair records"):
        dms.backward(torch.zeros(3, 16, dtype=torch.uint8, device=dev),
                     torch.zeros(3, 2, device=dev), grad)
    with pytest.raises(ValueError, match="same shape"):
        dms.critical(dms.Gradient(torch.zeros(4, 5, 6, dtype=torch.uint8, device=dev),
                                  torch.zeros(4, 5, 7, dtype=torch.int64, device=dev),
                                  torch.zeros(4, dtype=torch.int64, device=dev)))
    with pytest.raises(ValueError, match="must be torch.float32"):
        dms.order(torch.zeros(4, 5, 6, dtype=torch.float64, device=dev))
