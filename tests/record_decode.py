"""Test-side decoder of the gradient records documented in include/dms.h.

Turns (desc, rec) into the canonical list of discrete vectors
(tail_dim, tail_id, head_id), sorted by (dim, tail), and the critical lists,
so that the CUDA output can be compared with the oracle's.  Written from the
header's description only, with its own lattice geometry.
"""
from __future__ import annotations

import itertools

import numpy as np

EDGE_C = [1, 2, 4, 3, 5, 6, 7]
TRI_PQ = [(1, 3), (2, 3), (1, 5), (4, 5), (2, 6), (4, 6),
          (1, 7), (2, 7), (4, 7), (3, 7), (5, 7), (6, 7)]
TET_C = [(1, 3), (1, 5), (2, 3), (2, 6), (4, 5), (4, 6)]


def cvec(c):
    return np.array([c & 1, (c >> 1) & 1, (c >> 2) & 1])


class Lattice:
    def __init__(self, nx, ny, nz):
        self.nx, self.ny, self.nz = nx, ny, nz

    def lin(self, p):
        return int(p[0] + self.nx * (p[1] + self.ny * p[2]))

    def pt(self, v):
        return np.array([v % self.nx, (v // self.nx) % self.ny, v // (self.nx * self.ny)])

    def simplex_id(self, pts):
        """id of the simplex on the unbounded lattice (anchor may lie outside)."""
        pts = [np.asarray(p) for p in pts]
        anchor = min(pts, key=lambda p: int(p.sum()))
        corners = sorted(int((p - anchor) @ np.array([1, 2, 4])) for p in pts if (p != anchor).any())
        d = len(pts) - 1
        if d == 1:
            k = EDGE_C.index(corners[0])
            return 7 * self.lin(anchor) + k
        if d == 2:
            return 12 * self.lin(anchor) + TRI_PQ.index(tuple(corners))
        return 6 * self.lin(anchor) + TET_C.index(tuple(corners[:2]))

    def edge_pts(self, a, k):
        p = self.pt(a)
        return [p, p + cvec(EDGE_C[k])]

    def tet_chain(self, a, k):
        p = self.pt(a)
        c1, c2 = TET_C[k]
        return [p, p + cvec(c1), p + cvec(c2), p + cvec(7)]

    def edge_cofacets(self, a, k):
        """ids of all triangles holding edge (a, k) on the unbounded lattice,
        increasing."""
        e0, e1 = self.edge_pts(a, k)
        out = []
        for u in itertools.product((-1, 0, 1), repeat=3):
            w = e0 + np.array(u)
            pts = [e0, e1, w]
            if (w == e0).all() or (w == e1).all():
                continue
            ok = True
            for p, q in itertools.combinations(pts, 2):
                dd = q - p
                if not (((dd >= 0) & (dd <= 1)).all() or ((dd <= 0) & (dd >= -1)).all()):
                    ok = False
            if ok:
                out.append(self.simplex_id(pts))
        return sorted(out)


def decode(desc: np.ndarray, rec: np.ndarray, nx: int, ny: int, nz: int):
    """Returns (pairs [k,3] int64 sorted by (dim, tail), crit lists per dim).

    Ids are linear in the anchor (id = t*anchor + type), so every relation is
    tabulated once at the origin of the unbounded lattice and shifted."""
    L = Lattice(nx, ny, nz)
    zero = np.zeros(3, dtype=np.int64)
    desc = desc.reshape(-1).astype(np.int64)
    rec = rec.reshape(-1).view(np.uint64).astype(np.uint64)
    n = nx * ny * nz
    v = np.arange(n, dtype=np.int64)
    assert ((desc < 14) | (desc == 15)).all()
    # vertex -> edge
    slot_off = [cvec(c) for c in EDGE_C] + [-cvec(c) for c in EDGE_C]
    edge_of_slot = np.array([L.simplex_id([zero, o]) for o in slot_off], dtype=np.int64)
    lo = desc < 14
    vp = np.stack([np.zeros(int(lo.sum()), np.int64), v[lo],
                   edge_of_slot[desc[lo]] + 7 * v[lo]], axis=1)
    crit = [v[desc == 15]]
    # edges
    ecodes = np.stack([(rec >> np.uint64(3 * k)) & np.uint64(7) for k in range(7)], 1).astype(np.int64)
    cof = [L.edge_cofacets(0, k) for k in range(7)]
    cof_tab = np.full((7, 7), -1, dtype=np.int64)
    for k in range(7):
        for j, t in enumerate(cof[k]):
            cof_tab[k, j + 1] = t
    a_idx, k_idx = np.nonzero((ecodes >= 1) & (ecodes <= 6))
    c = ecodes[a_idx, k_idx]
    assert (cof_tab[k_idx, c] != -1).all()
    ep = np.stack([np.ones_like(a_idx), 7 * a_idx + k_idx, cof_tab[k_idx, c] + 12 * a_idx], 1)
    ca, ck = np.nonzero(ecodes == 7)
    crit.append(np.sort(7 * ca + ck))
    # triangles
    tb = np.stack([(rec >> np.uint64(21 + k)) & np.uint64(1) for k in range(12)], 1).astype(bool)
    ta, tk = np.nonzero(tb)
    crit.append(np.sort(12 * ta + tk))
    # tetrahedra
    qcodes = np.stack([(rec >> np.uint64(33 + 3 * k)) & np.uint64(7) for k in range(6)], 1).astype(np.int64)
    fac_tab = np.full((6, 5), -1, dtype=np.int64)
    for k in range(6):
        chain = L.tet_chain(0, k)
        for i in range(4):
            fac_tab[k, i + 1] = L.simplex_id([q for j, q in enumerate(chain) if j != i])
    qa, qk = np.nonzero((qcodes >= 1) & (qcodes <= 4))
    qc = qcodes[qa, qk]
    tp = np.stack([np.full_like(qa, 2), fac_tab[qk, qc] + 12 * qa, 6 * qa + qk], 1)
    assert not ((qcodes == 5) | (qcodes == 6)).any()
    qa7, qk7 = np.nonzero(qcodes == 7)
    crit.append(np.sort(6 * qa7 + qk7))
    assert ((rec >> np.uint64(51)) == 0).all()
    pairs = np.concatenate([vp, ep, tp]).astype(np.int64)
    order = np.lexsort((pairs[:, 1], pairs[:, 0]))
    return pairs[order], [np.asarray(x, dtype=np.int64) for x in crit]
