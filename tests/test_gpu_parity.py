"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer, index and id outputs are compared bit-exactly; pair values are
copies of input floats, so they are compared bit-exactly too.  Sizes span
several CTA tiles (32 x 32 anchors) with ragged tails in every axis.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import record_decode as rd

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2505_21266_gb300 as dms
from paper_2505_21266_gb300 import fields


def _fields(shape, seed):
    rng = np.random.default_rng(seed)
    return {
        "uniform": rng.random(shape).astype(np.float32),
        "ties": rng.integers(0, 5, size=shape).astype(np.float32),
        "signed": rng.choice(np.array([-0.0, 0.0, 1.0, -1.0, np.inf, -np.inf, 2.5],
                                      dtype=np.float32), size=shape),
        "ramp": np.arange(int(np.prod(shape)), dtype=np.float32).reshape(shape),
        "reverse": np.arange(int(np.prod(shape)), dtype=np.float32)[::-1].reshape(shape).copy(),
        "mixture": fields.gaussian_mixture(shape, 6, (0.1, 0.3), 1e-3, seed).numpy(),
    }


def _run_gpu(f_np):
    f = torch.from_numpy(f_np).cuda()
    res = dms.diagram(f)
    torch.cuda.synchronize()
    return res


def _pairs_np(t, dtype=dms.PAIR_DTYPE):
    return t.cpu().numpy().view(dtype).reshape(-1)


def _check_all(f_np, r=None):
    nz, ny, nx = f_np.shape
    if r is None:
        r = oracle.run(f_np)
    g = _run_gpu(f_np)
    # (i) order
    assert np.array_equal(g.order.cpu().numpy().reshape(-1), r.order)
    # (ii) gradient: every discrete vector and every critical simplex
    desc = g.grad.desc.cpu().numpy()
    rec = g.grad.rec.cpu().numpy()
    pairs, crit = rd.decode(desc, rec, nx, ny, nz)
    assert np.array_equal(pairs, r.get(oracle.GRAD_PAIRS))
    counts = g.grad.counts.cpu().numpy()
    for d in range(4):
        assert np.array_equal(crit[d], r.crit(d))
        assert counts[d] == len(r.crit(d))
        # (iii) compaction
        assert np.array_equal(g.crit[d].cpu().numpy(), r.crit(d))
    # (iv) diagrams, values bit-exact; the library lists pairs by saddle id
    for mine, ref, key in ((g.diagrams.d0, oracle.D0, "death_id"),
                           (g.diagrams.d2, oracle.D2, "birth_id")):
        a = _pairs_np(mine)
        b = r.get(ref)
        b = b[np.argsort(b[key], kind="stable")]
        assert len(a) == len(b)
        for k in ("birth_id", "death_id", "birth_vtx", "death_vtx"):
            assert np.array_equal(a[k], b[k]), k
        for k in ("birth", "death"):
            assert np.array_equal(a[k].view(np.uint32), b[k].view(np.uint32)), k
    ess = _pairs_np(g.diagrams.d0_essential)
    ress = r.get(oracle.D0_ESSENTIAL)
    assert ess["birth_id"][0] == ress["birth_id"][0] and ess["death_id"][0] == -1
    assert np.isinf(ess["death"][0])


@pytest.mark.parametrize("shape", [(2, 2, 2), (3, 5, 4), (7, 9, 11), (17, 33, 35),
                                   (12, 70, 41), (40, 3, 66)])
def test_parity_small_shapes(shape):
    for name, f in _fields(shape, sum(shape)).items():
        _check_all(f)


def test_parity_config1_64cubed():
    """64^3 Gaussian mixture + U[0, 1e-3) (several tiles, two z-chunks)."""
    f = fields.config1(0).numpy()
    _check_all(f)


def test_parity_uniform_noise_40cubed():
    f = fields.uniform01((40, 41, 43), 11).numpy()
    _check_all(f)


def test_parity_quantized_noise():
    f = fields.quantized_noise((33, 34, 35), 256, 2).numpy()
    _check_all(f)


def test_order_large_ragged():
    """Order only, 1,000,001-ish vertices with a ragged last tile, ties."""
    rng = np.random.default_rng(7)
    f = rng.integers(0, 1000, size=(101, 99, 101)).astype(np.float32)
    o = dms.order(torch.from_numpy(f).cuda()).cpu().numpy().reshape(-1)
    g = f.ravel().copy()
    g[g == 0] = 0.0
    idx = np.argsort(g, kind="stable")
    ref = np.empty(g.size, dtype=np.int64)
    ref[idx] = np.arange(g.size)
    assert np.array_equal(o.astype(np.int64), ref)


def test_nan_is_reported():
    f = np.random.default_rng(0).random((8, 8, 8)).astype(np.float32)
    f[3, 4, 5] = np.nan
    with pytest.raises(dms.DMSError) as e:
        dms.order(torch.from_numpy(f).cuda())
    assert e.value.code == 3


def test_bad_dims_are_rejected():
    with pytest.raises(dms.DMSError) as e:
        dms.order(torch.zeros((1, 4, 4), dtype=torch.float32, device="cuda"))
    assert e.value.code == 2


def test_capacity_error_reports_counts():
    f = torch.from_numpy(fields.uniform01((10, 10, 10), 3).numpy()).cuda()
    g = dms.gradient(dms.order(f))
    need = [int(x) for x in g.counts.cpu()]
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    lists, counts = dms.critical(g, caps=[need[0], need[1] - 1, need[2], need[3]], status=st)
    torch.cuda.synchronize()
    assert int(st.item()) & (1 << 4)
    assert [int(x) for x in counts.cpu()] == need


def test_parity_structured_fields():
    """Plateaus and periodic patterns over several tiles and z-chunks: a
    constant field (every comparison decided by the vertex offset: one
    critical simplex, no pairs), stripes along one axis, and a checkerboard
    (a dense critical set: ~1/4 of the edges and triangles are critical)."""
    def grid(shape):
        return np.meshgrid(*[np.arange(s) for s in shape], indexing="ij")
    z, y, x = grid((36, 50, 70))
    const = np.zeros(z.shape, dtype=np.float32)
    stripes = ((x // 3) % 4).astype(np.float32) - 1.5
    z, y, x = grid((18, 34, 40))
    checker = ((x + y + z) % 2).astype(np.float32)
    for f in (const, stripes, checker):
        _check_all(np.ascontiguousarray(f))
    r = oracle.run(const)
    assert [len(r.crit(d)) for d in range(4)] == [1, 0, 0, 0]


def test_stream_of_host_fields_matches_one_by_one():
    """diagrams_from_host (the next field's copy overlapped with the current
    field's path, two device buffers) gives each field the pairs it gets
    alone, also when shapes change along the stream."""
    xs = [fields.gaussian_mixture((20, 21, 22), 5, (0.1, 0.3), 1e-3, s).numpy() for s in range(3)]
    xs.append(np.random.default_rng(4).random((9, 30, 17)).astype(np.float32))
    hosts = [torch.from_numpy(x).pin_memory() for x in xs]
    got = list(dms.diagrams_from_host(hosts))
    assert len(got) == len(xs)
    for (d0, d2, ess), x in zip(got, xs):
        r = oracle.run(x)
        for mine, ref, key in ((d0, oracle.D0, "death_id"), (d2, oracle.D2, "birth_id")):
            b = r.get(ref)
            b = b[np.argsort(b[key], kind="stable")]
            assert mine.tobytes() == b.tobytes()
        assert ess["birth_id"][0] == r.get(oracle.D0_ESSENTIAL)["birth_id"][0]


def test_stream_reports_a_nan_field():
    """In a stream of host fields the order's NaN check is read after the
    gradient kernel is queued (the sort flags a NaN and still writes a
    permutation); a NaN in the second field still raises the order's error,
    before the first field's arrays, which come after the second's path."""
    good = fields.gaussian_mixture((12, 13, 14), 4, (0.1, 0.3), 1e-3, 0).numpy()
    bad = good.copy()
    bad[5, 6, 7] = np.nan
    out = []
    with pytest.raises(dms.DMSError) as e:
        for res in dms.diagrams_from_host([torch.from_numpy(good).pin_memory(),
                                           torch.from_numpy(bad).pin_memory()]):
            out.append(res)
    assert e.value.code == 3
    assert len(out) == 0  # the first field's arrays come after the second's path
