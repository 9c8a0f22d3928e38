"""Independent, test-side restatement of the Freudenthal (Kuhn) complex of a
3D grid and of the persistence computations that pin the oracle.

Written from the definitions only (Sec. 2.1 triangulation and lexicographic
filtration, Sec. 2.4-2.5 persistence pairs), without reference to the oracle's
or the CUDA library's code:

* the complex is generated as the set of all faces of the six tetrahedra of
  every cube (the cube split along its (1,1,1) diagonal, each tet a chain of
  corners under the componentwise order);
* simplices are sorted vertex tuples; the id convention of the library is
  recomputed here from its documented type tables (anchor = componentwise
  smallest vertex);
* persistence pairs come from union-find over all edges (Kruskal, elder
  rule), from union-find over tetrahedra plus an outside node (the dual
  graph), and from a plain Z2 boundary-matrix reduction.
"""
from __future__ import annotations

import itertools

import numpy as np

# documented type tables: corner bit 0 = +x, bit 1 = +y, bit 2 = +z
EDGE_TYPES = [(1,), (2,), (4,), (3,), (5,), (6,), (7,)]
TRI_TYPES = [(1, 3), (2, 3), (1, 5), (4, 5), (2, 6), (4, 6),
             (1, 7), (2, 7), (4, 7), (3, 7), (5, 7), (6, 7)]
TET_TYPES = [(1, 3, 7), (1, 5, 7), (2, 3, 7), (2, 6, 7), (4, 5, 7), (4, 6, 7)]
TYPE_TABLES = {1: EDGE_TYPES, 2: TRI_TYPES, 3: TET_TYPES}
NTYPES = {0: 1, 1: 7, 2: 12, 3: 6}


class Complex:
    def __init__(self, nx: int, ny: int, nz: int):
        self.nx, self.ny, self.nz = nx, ny, nz
        self.n = nx * ny * nz
        simplices = set()
        for z in range(nz - 1):
            for y in range(ny - 1):
                for x in range(nx - 1):
                    for perm in itertools.permutations(range(3)):
                        p = [x, y, z]
                        chain = [self.vid(*p)]
                        for ax in perm:
                            p[ax] += 1
                            chain.append(self.vid(*p))
                        for k in range(1, 5):
                            for sub in itertools.combinations(chain, k):
                                simplices.add(tuple(sorted(sub)))
        self.by_dim = {d: sorted(s for s in simplices if len(s) == d + 1) for d in range(4)}
        self._id = {}
        self._vs = {}
        for d in range(4):
            for s in self.by_dim[d]:
                i = self.type_id(s)
                self._id[s] = i
                self._vs[(d, i)] = s

    def vid(self, x, y, z):
        return x + self.nx * (y + self.ny * z)

    def xyz(self, v):
        return v % self.nx, (v // self.nx) % self.ny, v // (self.nx * self.ny)

    def type_id(self, s):
        d = len(s) - 1
        if d == 0:
            return s[0]
        cs = [self.xyz(v) for v in s]
        anchor = min(cs, key=sum)
        corners = []
        for c in cs:
            off = tuple(c[i] - anchor[i] for i in range(3))
            assert all(o in (0, 1) for o in off), s
            m = off[0] | (off[1] << 1) | (off[2] << 2)
            if m:
                corners.append(m)
        k = TYPE_TABLES[d].index(tuple(sorted(corners)))
        return self.vid(*anchor) * NTYPES[d] + k

    def id_of(self, s):
        return self._id[tuple(sorted(s))]

    def verts(self, d, i):
        return self._vs[(d, i)]

    def exists(self, d, i):
        return (d, i) in self._vs

    def facets(self, s):
        return [tuple(f) for f in itertools.combinations(s, len(s) - 1)] if len(s) > 1 else []

    def key(self, s, order):
        """Vertex orders by decreasing value (Python tuples compare
        lexicographically with a proper prefix first)."""
        return tuple(sorted((int(order[v]) for v in s), reverse=True))

    def max_vertex(self, s, order):
        return max(s, key=lambda v: order[v])

    def cofacets_of_triangle(self, s):
        s = set(s)
        return [t for t in self.by_dim[3] if s <= set(t)]

    def neighbours(self, v):
        out = set()
        for e in self.by_dim[1]:
            if v in e:
                out.add(e[0] if e[1] == v else e[1])
        return out


def canonical_order(field: np.ndarray) -> np.ndarray:
    """order[v] = rank of v in the stable sort of f (-0.0 == +0.0), via
    numpy's stable argsort -- the library-routine special case of Sec. 2.1."""
    f = np.ascontiguousarray(field, dtype=np.float32).ravel().copy()
    f[f == 0] = 0.0
    idx = np.argsort(f, kind="stable")
    order = np.empty(f.size, dtype=np.int64)
    order[idx] = np.arange(f.size)
    return order


class UnionFind:
    def __init__(self, elder):
        self.parent = {}
        self.elder = elder  # elder(a, b) -> the survivor

    def find(self, a):
        self.parent.setdefault(a, a)
        while self.parent[a] != a:
            self.parent[a] = self.parent[self.parent[a]]
            a = self.parent[a]
        return a


def kruskal_d0(cx: Complex, order):
    """All persistence pairs of dimension 0 of the lexicographic filtration:
    edges in increasing key order, components represented by their lowest
    vertex, the younger (higher) one dies.  Returns [(dying_vertex, edge)]."""
    uf = UnionFind(None)
    pairs = []
    for e in sorted(cx.by_dim[1], key=lambda s: cx.key(s, order)):
        a, b = uf.find(e[0]), uf.find(e[1])
        if a == b:
            continue
        if order[a] < order[b]:
            a, b = b, a
        pairs.append((a, e))
        uf.parent[a] = b
    return pairs


OUT = "OUT"


def dual_kruskal_d2(cx: Complex, order):
    """All persistence pairs of dimension 2 from the dual graph: tetrahedra
    plus one outside node, triangles visited in decreasing key order, the
    component with the lower maximum (outside = highest) dies.
    Returns [(triangle, dying_tet)]."""
    cof = {}
    for t in cx.by_dim[3]:
        for f in cx.facets(t):
            cof.setdefault(f, []).append(t)
    uf = UnionFind(None)

    def higher(a, b):
        if a == OUT:
            return True
        if b == OUT:
            return False
        return cx.key(a, order) > cx.key(b, order)

    pairs = []
    for s in sorted(cx.by_dim[2], key=lambda s: cx.key(s, order), reverse=True):
        ends = cof[s] + [OUT] * (2 - len(cof[s]))
        a, b = uf.find(ends[0]), uf.find(ends[1])
        if a == b:
            continue
        if higher(a, b):
            a, b = b, a
        pairs.append((s, a))
        uf.parent[a] = b
    return pairs


def reduction_pairs(cx: Complex, order):
    """Plain Z2 column reduction of the boundary matrix of the lexicographic
    filtration (columns as Python int bitsets).  Returns (pairs, essential):
    pairs = [(birth_simplex, death_simplex)], essential = [simplex]."""
    allsx = [s for d in range(4) for s in cx.by_dim[d]]
    allsx.sort(key=lambda s: cx.key(s, order))
    pos = {s: i for i, s in enumerate(allsx)}
    pivot = {}
    cols = {}
    pairs = []
    births = set()
    for j, s in enumerate(allsx):
        col = 0
        for f in cx.facets(s):
            col ^= 1 << pos[f]
        while col and (col.bit_length() - 1) in pivot:
            col ^= cols[pivot[col.bit_length() - 1]]
        if col:
            low = col.bit_length() - 1
            pivot[low] = j
            cols[j] = col
            pairs.append((allsx[low], s))
            births.add(low)
    deaths = {pos[b] for _, b in pairs}
    essential = [allsx[i] for i in range(len(allsx)) if i not in births and i not in deaths]
    return pairs, essential


def gf2_rank(m: np.ndarray) -> int:
    m = (np.asarray(m) & 1).astype(np.uint8).copy()
    rows, cols = m.shape
    r = 0
    for c in range(cols):
        piv = None
        for i in range(r, rows):
            if m[i, c]:
                piv = i
                break
        if piv is None:
            continue
        m[[r, piv]] = m[[piv, r]]
        for i in range(rows):
            if i != r and m[i, c]:
                m[i] ^= m[r]
        r += 1
        if r == rows:
            break
    return r


def lower_link_reduced_betti(cx: Complex, order, v, star):
    """Reduced Z2 Betti numbers (b~_-1, b~_0, b~_1, b~_2) of the lower link of
    v: the link simplices whose vertices all precede v."""
    low = lambda s: all(order[u] < order[v] for u in s)
    link = {d: [] for d in range(3)}
    for d in (1, 2, 3):
        for s in star[d]:
            rest = tuple(u for u in s if u != v)
            if low(rest):
                link[d - 1].append(rest)
    n = [len(link[d]) for d in range(3)]
    if n[0] == 0:
        return (1, 0, 0, 0)
    idx = [{s: i for i, s in enumerate(link[d])} for d in range(3)]
    # augmented chain complex: C2 -> C1 -> C0 -> Z2
    r0 = 1  # rank of the augmentation C0 -> Z2
    b1 = np.zeros((n[0], n[1]), dtype=np.uint8)
    for j, s in enumerate(link[1]):
        for f in cx.facets(s):
            b1[idx[0][f], j] = 1
    b2 = np.zeros((n[1], n[2]), dtype=np.uint8)
    for j, s in enumerate(link[2]):
        for f in cx.facets(s):
            b2[idx[1][f], j] = 1
    r1 = gf2_rank(b1) if n[1] else 0
    r2 = gf2_rank(b2) if n[2] else 0
    bt0 = n[0] - r0 - r1
    bt1 = n[1] - r1 - r2
    bt2 = n[2] - r2
    return (0, bt0, bt1, bt2)
