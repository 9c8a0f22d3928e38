"""The gradient record format of include/dms.h, checked on the CPU.

The oracle's gradient is written into the documented record layout by a
test-side encoder and read back by the test-side decoder used in the GPU
parity tests; the round trip must reproduce the oracle's pairs and critical
lists exactly.  This pins the decoder (and the documented layout) before any
GPU output goes through it.
"""
import numpy as np
import pytest

import oracle
import record_decode as rd


def encode_from_oracle(r, nx, ny, nz):
    L = rd.Lattice(nx, ny, nz)
    n = nx * ny * nz
    zero = np.zeros(3, dtype=np.int64)
    slot_off = [rd.cvec(c) for c in rd.EDGE_C] + [-rd.cvec(c) for c in rd.EDGE_C]
    edge_of_slot = {L.simplex_id([zero, o]): s for s, o in enumerate(slot_off)}
    p0, p1, p2, p3 = (r.partner(d) for d in range(4))
    desc = np.zeros(n, dtype=np.uint8)
    rec = np.zeros(n, dtype=np.uint64)
    for v in range(n):
        p = int(p0[v])
        if p == oracle.CRITICAL:
            desc[v] = 15
        else:
            desc[v] = edge_of_slot[(p >> 1) - 7 * v]
    cof = [L.edge_cofacets(0, k) for k in range(7)]
    for e in range(7 * n):
        p = int(p1[e])
        a, k = divmod(e, 7)
        if p == oracle.CRITICAL:
            code = 7
        elif p >= 0 and (p & 1):
            code = 1 + cof[k].index((p >> 1) - 12 * a)
        else:
            code = 0
        rec[a] |= np.uint64(code << (3 * k))
    for t in range(12 * n):
        if int(p2[t]) == oracle.CRITICAL:
            a, k = divmod(t, 12)
            rec[a] |= np.uint64(1 << (21 + k))
    for q in range(6 * n):
        p = int(p3[q])
        a, k = divmod(q, 6)
        if p == oracle.ABSENT:
            continue
        if p == oracle.CRITICAL:
            code = 7
        else:
            chain = L.tet_chain(a, k)
            facet = p >> 1
            code = None
            for i in range(4):
                if L.simplex_id([c for j, c in enumerate(chain) if j != i]) == facet:
                    code = i + 1
            assert code is not None
        rec[a] |= np.uint64(code << (33 + 3 * k))
    return desc, rec


@pytest.mark.parametrize("shape", [(2, 2, 2), (3, 4, 5), (6, 5, 7)])
def test_record_round_trip(rng, shape):
    for f in (rng.random(shape).astype(np.float32),
              rng.integers(0, 3, size=shape).astype(np.float32)):
        r = oracle.run(f, diagrams=False)
        nz, ny, nx = shape
        desc, rec = encode_from_oracle(r, nx, ny, nz)
        pairs, crit = rd.decode(desc, rec, nx, ny, nz)
        assert np.array_equal(pairs, r.get(oracle.GRAD_PAIRS))
        for d in range(4):
            assert np.array_equal(crit[d], r.crit(d))
