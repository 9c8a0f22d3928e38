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


def test_d1_properties_at_160_cubed_quantised_noise():
    """Beyond the oracle's reach, what holds at any size: every critical edge
    is in exactly one of D0 and D1, every critical triangle in exactly one
    of D1 and D2, the births are distinct, each death follows its birth in
    the filtration, and the values are the field's at the carriers."""
    f = fields.config2(0, "cuda", n=160)
    r = dms.diagram(f)
    d1 = dms.diagram_d1(f, r.order, r.grad, r.crit, r.diagrams)
    torch.cuda.synchronize()
    p = d1.cpu().numpy().view(dms.PAIR_DTYPE).reshape(-1)
    c1, c2 = r.crit[1].cpu().numpy(), r.crit[2].cpu().numpy()
    d0 = r.diagrams.numpy("d0")
    d2 = r.diagrams.numpy("d2")
    assert len(p) == len(c1) - len(d0) == len(c2) - len(d2)
    births = np.setdiff1d(c1, d0["death_id"])
    deaths = np.setdiff1d(c2, d2["birth_id"])
    assert np.array_equal(np.sort(p["birth_id"]), births)
    assert np.array_equal(p["death_id"], deaths)  # listed by increasing triangle id
    fl = f.cpu().numpy().reshape(-1)
    order = r.order.cpu().numpy().reshape(-1)
    assert np.array_equal(p["birth"].view(np.uint32), fl[p["birth_vtx"]].view(np.uint32))
    assert np.array_equal(p["death"].view(np.uint32), fl[p["death_vtx"]].view(np.uint32))
    assert np.all(order[p["death_vtx"]] >= order[p["birth_vtx"]])
