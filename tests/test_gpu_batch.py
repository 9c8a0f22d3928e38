"""The batched path (dms_batch_diagrams) against the oracle, field by field.

A batch of uneven fields -- noise, mixtures, ties, a 2x2x2 cube, thin slabs --
runs through one launch of the batched entry point; each field's pairs, ids
local to the field, must equal the oracle's for that field alone, bit for
bit.  The same holds for every gradient tile variant, for a CUDA-graph replay
on new inputs, and for the single-field path on the same fields.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2505_21266_gb300 as dms
from paper_2505_21266_gb300 import batch as B
from paper_2505_21266_gb300 import fields

SHAPES = [(5, 7, 9), (17, 13, 11), (2, 2, 2), (33, 40, 21), (64, 20, 3), (16, 16, 16),
          (3, 50, 70), (24, 24, 24)]


def _make(shapes, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i, s in enumerate(shapes):
        k = (i + seed) % 4
        if k == 0:
            x = rng.random(s).astype(np.float32)
        elif k == 1:
            x = rng.integers(0, 4, size=s).astype(np.float32)
        elif k == 2:
            x = fields.gaussian_mixture(s, 5, (0.1, 0.3), 1e-3, seed + i).numpy()
        else:
            x = rng.standard_normal(s).astype(np.float32)
        out.append(np.ascontiguousarray(x))
    return out


def _oracle_field(x):
    r = oracle.run(x)
    d0 = r.get(oracle.D0)
    d2 = r.get(oracle.D2)
    d0 = d0[np.argsort(d0["death_id"], kind="stable")]
    d2 = d2[np.argsort(d2["birth_id"], kind="stable")]
    return d0, d2, r.get(oracle.D0_ESSENTIAL)


def _same(a, b):
    assert len(a) == len(b)
    for k in ("birth_id", "death_id", "birth_vtx", "death_vtx"):
        assert np.array_equal(a[k].astype(np.int64), b[k].astype(np.int64)), k
    for k in ("birth", "death"):
        assert np.array_equal(a[k].view(np.uint32), b[k].view(np.uint32)), k


def _check_vs_oracle(res, xs):
    for (d0, d2, ess), x in zip(res, xs):
        r0, r2, ress = _oracle_field(x)
        _same(d0, r0)
        _same(d2, r2)
        assert ess["birth_id"][0] == ress["birth_id"][0] and ess["death_id"][0] == -1


def test_batch_matches_oracle_per_field():
    xs = _make(SHAPES, 1)
    b = B.Batch(SHAPES, "cuda")
    b.set_fields([torch.from_numpy(x) for x in xs])
    b.fit()
    torch.cuda.synchronize()
    _check_vs_oracle(b.results(), xs)
    # the order and records of each field are those of the field alone
    for i, x in enumerate(xs):
        r = oracle.run(x)
        o = b.order[b.offsets[i]:b.offsets[i + 1]].cpu().numpy()
        assert np.array_equal(o, r.order)


@pytest.mark.parametrize("variant", [1, 2, 3, 4, 5])
def test_tile_variants_agree(variant):
    """Every tile shape and lanes-per-vertex variant gives the same records
    and pairs as variant 0 (32 x 24 anchors, one lane per vertex)."""
    xs = _make(SHAPES, 2)
    ref = B.Batch(SHAPES, "cuda", tile_variant=0)
    ref.set_fields([torch.from_numpy(x) for x in xs])
    ref.fit()
    b = B.Batch(SHAPES, "cuda", tile_variant=variant)
    b.set_fields([torch.from_numpy(x) for x in xs])
    b.fit()
    torch.cuda.synchronize()
    assert torch.equal(ref.desc, b.desc) and torch.equal(ref.rec, b.rec)
    for (a0, a2, ae), (c0, c2, ce) in zip(ref.results(), b.results()):
        _same(a0, c0)
        _same(a2, c2)


def test_graph_replay_on_new_inputs():
    xs1, xs2 = _make(SHAPES, 3), _make(SHAPES, 4)
    b = B.Batch(SHAPES, "cuda")
    b.set_fields([torch.from_numpy(x) for x in xs1])
    # capacities that hold for both inputs (noise bound), then capture
    b.capture()
    b.set_fields([torch.from_numpy(x) for x in xs2])
    b.replay()
    torch.cuda.synchronize()
    _check_vs_oracle(b.results(), xs2)
    b.set_fields([torch.from_numpy(x) for x in xs1])
    b.replay()
    torch.cuda.synchronize()
    _check_vs_oracle(b.results(), xs1)


def test_batch_equals_per_field_path():
    shapes = fields.batch_shapes(12, 8, 48, seed=5)
    xs = [fields.batch_field(i, s, seed=5) for i, s in enumerate(shapes)]
    b = B.Batch(shapes, "cuda")
    b.set_fields(xs)
    b.fit()
    torch.cuda.synchronize()
    got = b.results()
    ref = B.per_field([x.cuda() for x in xs])
    for (a0, a2, ae), (c0, c2, ce) in zip(got, ref):
        _same(a0, c0)
        _same(a2, c2)
        assert ae["birth_id"][0] == ce["birth_id"][0]


def test_large_batch_order_and_pairs_equal_per_field():
    """A batch of at least 2^25 vertices builds its per-field orders by the
    bucketed inverse permutation (positions made local to each field on the
    way out); each field alone (under 2^25 vertices) uses the direct
    scatter.  Orders and pairs must agree field by field."""
    shapes = [(200, 230, 256), (190, 247, 251), (200, 250, 250)]  # 36,055,430 vertices
    assert sum(a * b * c for a, b, c in shapes) >= 1 << 25
    xs = [fields.batch_field(i, s, seed=9, device="cuda") for i, s in enumerate(shapes)]
    b = B.Batch(shapes, "cuda")
    b.set_fields(xs)
    b.fit()
    torch.cuda.synchronize()
    for i, x in enumerate(xs):
        mine = b.order[b.offsets[i]:b.offsets[i + 1]].view(torch.int32).reshape(x.shape)
        assert torch.equal(mine, dms.order(x).view(torch.int32))
    got = b.results()
    ref = B.per_field(xs)
    for (a0, a2, ae), (c0, c2, ce) in zip(got, ref):
        _same(a0, c0)
        _same(a2, c2)
        assert ae["birth_id"][0] == ce["birth_id"][0]
    del b, xs
    torch.cuda.empty_cache()


def test_capacity_growth():
    xs = _make(SHAPES[:3], 6)
    b = B.Batch(SHAPES[:3], "cuda", caps=[1, 1, 1, 1])
    b.set_fields([torch.from_numpy(x) for x in xs])
    b.fit()
    torch.cuda.synchronize()
    _check_vs_oracle(b.results(), xs)
