"""Parity of the 2D CUDA path (dms2_* through the C ABI) with the 2D oracle:
order, every discrete vector and critical simplex (decoded from the records
as include/dms.h describes them), the three critical lists, and every D0 /
D1 pair with its float values, bit for bit.  Grids span several 64 x 16
tiles with ragged tails."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2505_21266_gb300 as dms
from paper_2505_21266_gb300 import fields


def _edge_id(nx, p, q):
    """id of the edge between grid points p, q (x, y), from the definitions."""
    a = min(p, q, key=lambda t: t[0] + t[1])
    b = q if a == p else p
    c = (b[0] - a[0]) | ((b[1] - a[1]) << 1)
    return 3 * (a[0] + nx * a[1]) + [1, 2, 3].index(c)


def decode2d(desc, rec, nx, ny):
    """(pairs [k,3] sorted by (dim, tail), [crit0, crit1, crit2]) from the
    2D records, written from the header's description."""
    desc = desc.reshape(-1).astype(np.int64)
    rec = rec.reshape(-1).view(np.uint16).astype(np.int64)
    corner = [(1, 0), (0, 1), (1, 1)]
    pairs, crit, tri_side = [], [[], [], []], []
    for v in range(nx * ny):
        x, y = v % nx, v // nx
        d = int(desc[v])
        if d == 15:
            crit[0].append(v)
        else:
            assert 0 <= d < 6
            c = corner[d % 3]
            q = (x + c[0], y + c[1]) if d < 3 else (x - c[0], y - c[1])
            pairs.append((0, v, _edge_id(nx, (x, y), q)))
        r = int(rec[v])
        assert r >> 15 == 0
        for k in range(3):
            code = (r >> (3 * k)) & 7
            e = 3 * v + k
            if code == 7:
                crit[1].append(e)
            elif code in (1, 2):
                # triangles holding edge k at (x, y) on the unbounded lattice, by id
                if k == 0:
                    cof = [2 * (v - nx) + 1, 2 * v]
                elif k == 1:
                    cof = [2 * (v - 1), 2 * v + 1]
                else:
                    cof = [2 * v, 2 * v + 1]
                pairs.append((1, e, sorted(cof)[code - 1]))
            else:
                assert code == 0
        for k in range(2):
            code = (r >> (9 + 3 * k)) & 7
            t = 2 * v + k
            if code == 7:
                crit[2].append(t)
            elif code:
                assert code in (1, 2, 3)
                chain = [(x, y), (x + 1, y) if k == 0 else (x, y + 1), (x + 1, y + 1)]
                rest = [p for i, p in enumerate(chain) if i != code - 1]
                tri_side.append((1, _edge_id(nx, rest[0], rest[1]), t))
    assert set(tri_side) == {p for p in pairs if p[0] == 1}  # both sides agree
    out = np.array(sorted(pairs), dtype=np.int64).reshape(-1, 3)
    return out, [np.array(sorted(c), dtype=np.int64) for c in crit]


def _check(f_np):
    ny, nx = f_np.shape
    r = oracle.run2(f_np)
    res = dms.diagram2d(torch.from_numpy(f_np).cuda())
    torch.cuda.synchronize()
    assert np.array_equal(res.order.cpu().numpy().reshape(-1), r.order)
    gp, crit = decode2d(res.grad.desc.cpu().numpy(), res.grad.rec.cpu().numpy(), nx, ny)
    assert np.array_equal(gp, r.get(oracle.GRAD_PAIRS2))
    for d in range(3):
        assert np.array_equal(crit[d], r.crit(d)), d
        assert np.array_equal(res.crit[d].cpu().numpy(), r.crit(d)), d
    for which, ref, key in (("d0", oracle.D0_2, "death_id"), ("d1", oracle.D1_2, "birth_id")):
        a = res.diagrams.numpy(which)
        b = r.get(ref)
        b = b[np.argsort(b[key], kind="stable")]
        assert len(a) == len(b), which
        for k in ("birth_id", "death_id", "birth_vtx", "death_vtx"):
            assert np.array_equal(a[k], b[k]), (which, k)
        for k in ("birth", "death"):
            assert np.array_equal(a[k].view(np.uint32), b[k].view(np.uint32)), (which, k)
    ess = res.diagrams.numpy("d0_essential")
    assert ess["birth_id"][0] == r.get(oracle.D0_ESSENTIAL2)["birth_id"][0]
    assert ess["death_id"][0] == -1


@pytest.mark.parametrize("shape", [(2, 2), (2, 9), (9, 2), (5, 7), (17, 65), (40, 130)])
def test_parity_2d_small(shape):
    rng = np.random.default_rng(sum(shape))
    for f in (rng.random(shape).astype(np.float32),
              rng.integers(0, 4, size=shape).astype(np.float32),
              rng.choice(np.array([-0.0, 0.0, 1.0, -1.0, np.inf, -np.inf], dtype=np.float32),
                         size=shape),
              np.arange(int(np.prod(shape)), dtype=np.float32).reshape(shape)):
        _check(np.ascontiguousarray(f))


def test_parity_2d_mixture_and_noise():
    g = fields.gaussian_mixture((1, 200, 300), 12, (0.05, 0.2), 1e-3, 3).numpy()[0]
    _check(np.ascontiguousarray(g))
    q = fields.quantized_noise((1, 256, 256), 256, 4).numpy()[0]
    _check(np.ascontiguousarray(q))


def test_2d_errors():
    f = torch.zeros((1, 5), device="cuda")
    with pytest.raises(ValueError):
        dms.diagram2d(f[0])
    with pytest.raises(dms.DMSError):
        dms.order2d(f)  # a 1 x 5 grid
    g = torch.tensor([[0.0, float("nan")], [1.0, 2.0]], device="cuda")
    with pytest.raises(dms.DMSError):
        dms.order2d(g)


def test_parity_2d_1024_squared():
    """The 2D benchmark recipe (64 Gaussians, sigma U[0.01,0.1], + U[0,1e-2))
    at 1024^2 against the full 2D oracle: order, critical lists, every D0 /
    D1 pair and its values."""
    g = np.ascontiguousarray(
        fields.gaussian_mixture((1, 1024, 1024), 64, (0.01, 0.1), 1e-2, 0).numpy()[0])
    r = oracle.run2(g)
    res = dms.diagram2d(torch.from_numpy(g).cuda())
    torch.cuda.synchronize()
    assert np.array_equal(res.order.cpu().numpy().reshape(-1), r.order)
    for d in range(3):
        assert np.array_equal(res.crit[d].cpu().numpy(), r.crit(d)), d
    for which, ref, key in (("d0", oracle.D0_2, "death_id"), ("d1", oracle.D1_2, "birth_id")):
        a = res.diagrams.numpy(which)
        b = r.get(ref)
        b = b[np.argsort(b[key], kind="stable")]
        assert len(a) == len(b)
        for k in ("birth_id", "death_id", "birth_vtx", "death_vtx"):
            assert np.array_equal(a[k], b[k]), (which, k)
        for k in ("birth", "death"):
            assert np.array_equal(a[k].view(np.uint32), b[k].view(np.uint32)), (which, k)
