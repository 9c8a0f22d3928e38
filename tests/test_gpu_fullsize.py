"""Parity at full size: the 1024^3 Gaussian-mixture workload and the 512^3
quantised-noise workload, through the same calls the benchmark times.

The full oracle cannot run at these sizes, so the checks are
  * the order: a permutation that sorts (f with -0 == +0, offset), checked
    over all vertices; a few ranks recounted on the host;
  * the gradient and the critical simplices at sampled vertices: the
    oracle's ProcessLowerStars of each sampled vertex, computed from the
    field of the 5x5x5 block around it (ranks in the block order like the
    global order), against the records the GPU wrote for that lower star;
  * the diagrams: counts and structure over all pairs (one pair per minimum
    but the essential one, one per maximum, values copied from the field),
    and the elder rule at sampled pairs and at sampled critical edges and
    triangles, by the oracle's local component growth from the field.
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

TYPES = (1, 7, 12, 6)


@pytest.fixture(scope="module", params=["gaussian_1024", "quantized_512"])
def full(request):
    if request.param == "gaussian_1024":
        f = fields.config3(0, device="cuda")
    else:
        f = fields.config2(0, device="cuda")
    torch.cuda.synchronize()
    res = dms.diagram(f)
    torch.cuda.synchronize()
    nz, ny, nx = f.shape
    data = {
        "name": request.param, "dims": (nx, ny, nz), "f_dev": f, "res": res,
        "f": f.cpu().numpy(),
        "desc": res.grad.desc.cpu().numpy(),
        "rec": res.grad.rec.cpu().numpy(),
        "crit": [c.cpu().numpy() for c in res.crit],
        "d0": res.diagrams.numpy("d0"),
        "d2": res.diagrams.numpy("d2"),
        "ess": res.diagrams.numpy("d0_essential"),
    }
    yield data
    del data, res, f
    torch.cuda.empty_cache()


def test_order_is_the_stable_sort(full):
    f = full["f_dev"].reshape(-1)
    o = full["res"].order.reshape(-1).to(torch.int64)
    n = f.numel()
    assert int(o.min()) == 0 and int(o.max()) == n - 1
    inv = torch.full((n,), -1, dtype=torch.int64, device=f.device)
    inv[o] = torch.arange(n, device=f.device)
    assert bool((inv >= 0).all())  # every position taken once: a permutation
    key = f[inv] + 0.0  # -0.0 folds onto +0.0
    up = (key[1:] > key[:-1]) | ((key[1:] == key[:-1]) & (inv[1:] > inv[:-1]))
    assert bool(up.all())
    del inv, key, up
    # a few ranks recounted on the host from the definition
    fh = full["f"].reshape(-1) + np.float32(0.0)
    oh = full["res"].order.reshape(-1)
    rng = np.random.default_rng(7)
    for v in rng.integers(0, n, 3):
        fv = fh[v]
        rank = int(np.count_nonzero(fh < fv)) + int(np.count_nonzero(fh[:v] == fv))
        assert int(oh[v]) == rank


def _samples(dims, count, seed):
    nx, ny, nz = dims
    rng = np.random.default_rng(seed)
    pts = [(x, y, z) for x in (0, nx - 1) for y in (0, ny - 1) for z in (0, nz - 1)]
    pts += [(int(rng.integers(nx)), int(rng.integers(ny)), z) for z in (0, nz - 1) for _ in range(8)]
    pts += [(0, int(rng.integers(ny)), int(rng.integers(nz))) for _ in range(8)]
    pts += [tuple(int(rng.integers(n)) for n in dims) for _ in range(count)]
    return pts


def _global_id(d, crop_id, lo, cdims, dims):
    cx, cy, _ = cdims
    a, k = divmod(int(crop_id), TYPES[d])
    x, y, z = a % cx, (a // cx) % cy, a // (cx * cy)
    gx, gy, gz = x + lo[0], y + lo[1], z + lo[2]
    nx, ny, _ = dims
    return TYPES[d] * (gx + nx * (gy + ny * gz)) + k


def test_gradient_and_critical_at_sampled_vertices(full):
    nx, ny, nz = full["dims"]
    F, D, R = full["f"], full["desc"], full["rec"]
    crit = full["crit"]
    checked = 0
    for (x, y, z) in _samples(full["dims"], 400, 11):
        lo = (max(x - 2, 0), max(y - 2, 0), max(z - 2, 0))
        hi = (min(x + 3, nx), min(y + 3, ny), min(z + 3, nz))
        sl = (slice(lo[2], hi[2]), slice(lo[1], hi[1]), slice(lo[0], hi[0]))
        fc = np.ascontiguousarray(F[sl])
        dc = D[sl].copy()
        rcrop = R[sl].copy()
        cz, cy, cx = fc.shape
        # keep only the records of anchors in the 2x2x2 block of cubes at the
        # vertex: every simplex of its lower star is anchored there
        keep = np.zeros(fc.shape, dtype=bool)
        keep[max(z - 1, 0) - lo[2]:z - lo[2] + 1, max(y - 1, 0) - lo[1]:y - lo[1] + 1,
             max(x - 1, 0) - lo[0]:x - lo[0] + 1] = True
        rcrop[~keep] = 0
        dc[~keep] = 15
        vloc = (x - lo[0]) + cx * ((y - lo[1]) + cy * (z - lo[2]))
        gp, gcrit = rd.decode(dc, rcrop, cx, cy, cz)
        op, ocrit = oracle.lower_star_vertex(fc, vloc)
        star = {(int(d), int(t)) for d, t, _ in op} | {(int(d) + 1, int(h)) for d, _, h in op} | \
               {(int(d), int(s)) for d, s in ocrit}
        mine = {(int(d), int(t), int(h)) for d, t, h in gp
                if (int(d), int(t)) in star or (int(d) + 1, int(h)) in star}
        assert mine == {(int(d), int(t), int(h)) for d, t, h in op}, (x, y, z)
        mine_c = {(d, int(s)) for d in range(4) for s in gcrit[d] if (d, int(s)) in star}
        assert mine_c == {(int(d), int(s)) for d, s in ocrit}, (x, y, z)
        # the compaction lists hold exactly the critical simplices of the star
        cdims = (cx, cy, cz)
        for d, s in star:
            gid = _global_id(d, s, lo, cdims, (nx, ny, nz))
            j = np.searchsorted(crit[d], gid)
            listed = j < len(crit[d]) and crit[d][j] == gid
            assert listed == ((d, s) in mine_c), (x, y, z, d)
        checked += 1
    assert checked >= 400


def test_critical_counts(full):
    c = [len(x) for x in full["crit"]]
    assert c[0] - c[1] + c[2] - c[3] == 1  # Euler characteristic of a ball
    assert [int(v) for v in full["res"].grad.counts.cpu()] == c
    for lst in full["crit"]:
        assert np.all(np.diff(lst) > 0)


def _members(sorted_list, ids):
    j = np.searchsorted(sorted_list, ids)
    return (j < len(sorted_list)) & (sorted_list[np.minimum(j, len(sorted_list) - 1)] == ids)


def test_diagram_structure(full):
    F = full["f"].reshape(-1)
    crit = full["crit"]
    d0, d2, ess = full["d0"], full["d2"], full["ess"]
    assert len(d0) == len(crit[0]) - 1 and len(d2) == len(crit[3])
    births = np.sort(np.concatenate([d0["birth_id"], ess["birth_id"]]))
    assert np.array_equal(births, crit[0])
    assert np.all(np.diff(d0["death_id"]) > 0)
    assert np.all(_members(crit[1], d0["death_id"]))
    assert np.array_equal(np.sort(d2["death_id"]), crit[3])
    assert np.all(np.diff(d2["birth_id"]) > 0)
    assert np.all(_members(crit[2], d2["birth_id"]))
    for p in (d0, d2):
        assert np.array_equal(p["birth"].view(np.uint32), F[p["birth_vtx"]].view(np.uint32))
        assert np.array_equal(p["death"].view(np.uint32), F[p["death_vtx"]].view(np.uint32))
        assert np.all(p["death"] >= p["birth"])
    assert ess["death_id"][0] == -1 and np.isinf(ess["death"][0])
    assert F[ess["birth_id"][0]] == F.min()


def test_elder_rule_at_sampled_pairs_and_saddles(full):
    f = full["f"]
    d0, d2, crit = full["d0"], full["d2"], full["crit"]
    rng = np.random.default_rng(13)
    decided = 0
    # sampled D0 pairs: the edge kills exactly the recorded minimum
    for i in rng.choice(len(d0), 40, replace=False):
        st, dying = oracle.d0_edge_local(f, int(d0["death_id"][i]), limit=1_000_000)
        assert st != 0
        if st == 1:
            assert dying == int(d0["birth_id"][i])
            decided += 1
    # sampled critical edges: a death in D0 iff the elder rule says so
    for e in rng.choice(crit[1], 40, replace=False):
        st, dying = oracle.d0_edge_local(f, int(e), limit=1_000_000)
        j = np.searchsorted(d0["death_id"], e)
        there = j < len(d0) and d0["death_id"][j] == e
        if st == 1:
            assert there and int(d0["birth_id"][j]) == dying
            decided += 1
        elif st == 0:
            assert not there
            decided += 1
    # the same on the dual side
    for i in rng.choice(len(d2), 25, replace=False):
        st, dying = oracle.d2_triangle_local(f, int(d2["birth_id"][i]), limit=100_000)
        assert st != 0
        if st == 1:
            assert dying == int(d2["death_id"][i])
            decided += 1
    for t in rng.choice(crit[2], 25, replace=False):
        st, dying = oracle.d2_triangle_local(f, int(t), limit=100_000)
        j = np.searchsorted(d2["birth_id"], t)
        there = j < len(d2) and d2["birth_id"][j] == t
        if st == 1:
            assert there and int(d2["death_id"][j]) == dying
            decided += 1
        elif st == 0:
            assert not there
            decided += 1
    assert decided >= 60
