"""Parity at the workloads' own shapes, and the pairing's round bounds.

* The differentiable workload's field (128^3, 32 Gaussians + U[0,1e-4)) through
  the whole single-field path against the full oracle: order, every discrete
  vector, the critical lists and every pair, bit for bit.
* The batched workload's recipe (axes U{32..256}, even fields Gaussian
  mixtures, odd fields U[0,1)) on those of its first shapes that the oracle
  finishes in about a minute, in one batched launch, against the oracle field
  by field (the oracle runs in a spawned process pool on the host cores).
* A chain of wells whose barriers rise and whose minima deepen along x: the
  exact pairing rounds merge one saddle per round there.  The single-field
  path must hand such a chain to its sorted finish after a bounded number of
  rounds, and the batched path, whose exact rounds are a fixed number, must
  finish what they leave (more than its one-CTA finish holds) in order.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import oracle_jobs
import record_decode as rd

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2505_21266_gb300 as dms
from paper_2505_21266_gb300 import _lib, fields
from paper_2505_21266_gb300 import batch as B

def _same_pairs(a, b):
    assert len(a) == len(b)
    for k in ("birth_id", "death_id", "birth_vtx", "death_vtx"):
        assert np.array_equal(a[k].astype(np.int64), b[k].astype(np.int64)), k
    for k in ("birth", "death"):
        assert np.array_equal(a[k].view(np.uint32), b[k].view(np.uint32)), k


def test_differentiable_workload_field_full_parity():
    f_np = fields.config4(0).numpy()
    r = oracle.run(f_np)
    g = dms.diagram(torch.from_numpy(f_np).cuda())
    torch.cuda.synchronize()
    nz, ny, nx = f_np.shape
    assert np.array_equal(g.order.cpu().numpy().reshape(-1), r.order)
    pairs, crit = rd.decode(g.grad.desc.cpu().numpy(), g.grad.rec.cpu().numpy(), nx, ny, nz)
    assert np.array_equal(pairs, r.get(oracle.GRAD_PAIRS))
    for d in range(4):
        assert np.array_equal(crit[d], r.crit(d))
        assert np.array_equal(g.crit[d].cpu().numpy(), r.crit(d))
    d0, d2, ess = oracle_jobs.sorted_pairs(r)
    _same_pairs(g.diagrams.numpy("d0"), d0)
    _same_pairs(g.diagrams.numpy("d2"), d2)
    mine = g.diagrams.numpy("d0_essential")
    assert mine["birth_id"][0] == ess["birth_id"][0] and mine["death_id"][0] == -1


def _batch_subset(max_vertices=1_300_000, first=40):
    shapes = fields.batch_shapes(256, 32, 256, seed=0)[:first]
    return [(i, s) for i, s in enumerate(shapes) if s[0] * s[1] * s[2] <= max_vertices]


def test_batched_workload_shapes_against_oracle():
    picked = _batch_subset()
    assert len(picked) >= 10
    ncpu = max(1, min(len(picked), (os.cpu_count() or 2) - 1))
    with oracle_jobs.pool(ncpu) as pool:
        jobs = [pool.apply_async(oracle_jobs.batch_field_oracle, (i, s, 0)) for i, s in picked]
        shapes = [s for _, s in picked]
        b = B.Batch(shapes, "cuda")
        b.set_fields([fields.batch_field(i, s, seed=0) for i, s in picked])
        b.fit()
        torch.cuda.synchronize()
        got = b.results()
        refs = [j.get(timeout=1800) for j in jobs]
    for k, ((i, s), (d0, d2, ess), ref) in enumerate(zip(picked, got, refs)):
        a, z = int(b.offsets[k]), int(b.offsets[k + 1])
        assert np.array_equal(b.order[a:z].cpu().numpy(), ref["order"]), (i, s)
        _same_pairs(d0, ref["d0"])
        _same_pairs(d2, ref["d2"])
        assert ess["birth_id"][0] == ref["ess"]["birth_id"][0]
    counts = b.counts.cpu().numpy()
    for d in range(4):
        assert counts[d] == sum(len(ref["crit"][d]) for ref in refs)


def chain_field(n_wells: int, deeper_right: bool = True) -> np.ndarray:
    """[2, 2, 4 n + 1] field constant across y, z: well i at x = 4i + 2 with
    value -i (deeper along x; i / 4, shallower, when not deeper_right), the
    barrier before it at x = 4i with value i + 1/2 (higher along x),
    midpoints in between.  Alg. 1 merges the wells from the left one by one;
    with deeper_right the exact rounds merge one saddle per round, without it
    they merge every saddle in the first round."""
    nx = 4 * n_wells + 1
    g = np.empty(nx, np.float64)
    for x in range(nx):
        i, r = divmod(x, 4)
        well = -float(i) if deeper_right else 0.25 * i
        g[x] = i + 0.5 if r == 0 else (well if r == 2 else np.nan)
    for x in range(nx):
        if np.isnan(g[x]):
            g[x] = 0.5 * (g[x - 1] + g[x + 1])
    return np.ascontiguousarray(np.broadcast_to(g.astype(np.float32), (2, 2, nx)))


def test_chain_of_wells_single_field_rounds_are_bounded():
    n = 3000
    f_np = chain_field(n)
    r = oracle.run(f_np)
    assert len(r.get(oracle.D0)) == n - 1
    lib = _lib.load()
    f = torch.from_numpy(f_np).cuda()
    o = dms.order(f)
    g = dms.gradient(o)
    c = dms.critical(g)
    torch.cuda.synchronize()
    before = lib.dms_launch_count()
    res = dms.diagram_d0d2(f, o, g, c)
    torch.cuda.synchronize()
    launches = lib.dms_launch_count() - before
    # Borůvka rounds (log2 of the wells) plus a few exact rounds and the
    # sorted finish; one launch pair per saddle would be ~6000
    assert launches < 200, launches
    d0, d2, _ = oracle_jobs.sorted_pairs(r)
    _same_pairs(res.numpy("d0"), d0)
    _same_pairs(res.numpy("d2"), d2)


def test_batch_finishes_beyond_its_round_budget():
    """A chain longer than the batch's fixed exact rounds plus its one-CTA
    finish (4096 saddles): the saddles still live are sorted on the device
    and finished in Alg. 1's order, so the pairs are the oracle's; the same
    buffers then take new inputs of the same shapes."""
    n = B._lib.load().dms_batch_max_rounds() + 4096 + 200
    chain = chain_field(n)
    small = fields.batch_field(0, (9, 10, 11), seed=3).numpy()
    shapes = [chain.shape, small.shape]
    b = B.Batch(shapes, "cuda")
    for x0 in (chain, chain_field(n, deeper_right=False)):
        b.set_fields([torch.from_numpy(x0), torch.from_numpy(small)])
        b.launch()
        torch.cuda.synchronize()
        assert b.status_code() == 0
        for (d0, d2, ess), x in zip(b.results(), (x0, small)):
            rr = oracle.run(x)
            r0, r2, re = oracle_jobs.sorted_pairs(rr)
            _same_pairs(d0, r0)
            _same_pairs(d2, r2)
            assert ess["birth_id"][0] == re["birth_id"][0]
