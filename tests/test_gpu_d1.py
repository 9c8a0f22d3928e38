"""D1 on the GPU (dms_diagram_d1: homologous propagation, Sec. 2.5, Alg. 2-3,
as bulk rounds over all columns) against the oracle's sequential Alg. 3,
which the CPU suite pins to a full boundary-matrix reduction: every pair's
edge and triangle ids, carrier vertices and value bits, on small grids with
ties, signed zeros, infinities, noise and mixtures, at the 64^3 and 128^3
workload fields, and with a pool small enough to force the boundaries to
grow (and, once, to run out)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2505_21266_gb300 as dms
from paper_2505_21266_gb300 import fields
from test_gpu_configs import _same_pairs
from test_gpu_parity import _fields


def _gpu_d1(f_np, pool_entries=0):
    f = torch.from_numpy(np.ascontiguousarray(f_np)).cuda()
    r = dms.diagram(f)
    d1 = dms.diagram_d1(f, r.order, r.grad, r.crit, r.diagrams, pool_entries=pool_entries)
    torch.cuda.synchronize()
    return d1.cpu().numpy().view(dms.PAIR_DTYPE).reshape(-1)


def _oracle_d1(f_np):
    r = oracle.run(f_np, d1=True)
    d1 = r.get(oracle.D1)
    return d1[np.argsort(d1["death_id"], kind="stable")]


@pytest.mark.parametrize("shape,seed", [((2, 2, 2), 0), ((9, 7, 11), 1), ((23, 37, 41), 2),
                                        ((40, 33, 35), 3)])
def test_d1_matches_oracle(shape, seed):
    for name, f_np in _fields(shape, seed).items():
        _same_pairs(_gpu_d1(f_np), _oracle_d1(f_np))


@pytest.mark.parametrize("which", ["c1_64", "noise_64", "c4_128"])
def test_d1_on_workload_fields(which):
    if which == "c1_64":
        f_np = fields.config1(0).numpy()
    elif which == "noise_64":
        f_np = fields.uniform01((64, 64, 64), 3).numpy()
    else:
        f_np = fields.config4(0).numpy()
    _same_pairs(_gpu_d1(f_np), _oracle_d1(f_np))


def test_d1_pool_too_small_then_grown():
    """A pool just above the first heap segments: boundaries must grow into
    it, some run out (DMS_ERR_CAPACITY, the stream left idle), and with a
    larger pool the pairs are the oracle's."""
    f_np = fields.uniform01((24, 26, 28), 5).numpy()
    ref = _oracle_d1(f_np)
    f = torch.from_numpy(f_np).cuda()
    r = dms.diagram(f)
    n2 = int(r.crit[2].numel())
    with pytest.raises(dms.DMSError) as ei:
        dms.diagram_d1(f, r.order, r.grad, r.crit, r.diagrams, pool_entries=16 * n2 + 64,
                       max_tries=1)
    torch.cuda.synchronize()
    assert ei.value.code == 4
    d1 = dms.diagram_d1(f, r.order, r.grad, r.crit, r.diagrams, pool_entries=16 * n2 + 64)
    torch.cuda.synchronize()
    _same_pairs(d1.cpu().numpy().view(dms.PAIR_DTYPE).reshape(-1), ref)
