"""Pins of the 2D oracle against what the mathematics fixes, with a test-side
restatement of the 2D Freudenthal complex (every square split along its
(1,1) diagonal; the two triangles are chains of square corners):

* order = numpy's stable argsort of the canonical key;
* the gradient: a matching whose pairs share their top vertex, acyclic;
  per vertex, the critical k-simplices of its lower star number the reduced
  Betti number b~_{k-1} of its lower link;
* #minima - #saddles + #maxima = 1 (Euler characteristic of a disk);
* D0 = Kruskal over all edges by increasing key (elder rule) without the
  zero-persistence pairs; D1 = the dual union-find over triangles plus the
  outside by decreasing edge key; every pair also = the Z2 boundary-matrix
  reduction's pairs whose simplices have different top vertices;
* ramps and constant fields have a single critical simplex.
"""
import itertools

import numpy as np
import pytest

import oracle

EDGE_T = [(1,), (2,), (3,)]
TRI_T = [(1, 3), (2, 3)]


class Complex2:
    def __init__(self, nx, ny):
        self.nx, self.ny = nx, ny
        sx = set()
        for y in range(ny - 1):
            for x in range(nx - 1):
                for first in ((1, 0), (0, 1)):
                    chain = [(x, y), (x + first[0], y + first[1]), (x + 1, y + 1)]
                    ids = [self.vid(*p) for p in chain]
                    for k in (1, 2, 3):
                        for sub in itertools.combinations(ids, k):
                            sx.add(tuple(sorted(sub)))
        self.by_dim = {d: sorted(s for s in sx if len(s) == d + 1) for d in range(3)}

    def vid(self, x, y):
        return x + self.nx * y

    def xy(self, v):
        return v % self.nx, v // self.nx

    def type_id(self, s):
        d = len(s) - 1
        if d == 0:
            return s[0]
        cs = [self.xy(v) for v in s]
        a = min(cs, key=sum)
        corners = sorted((c[0] - a[0]) | ((c[1] - a[1]) << 1) for c in cs if c != a)
        table = EDGE_T if d == 1 else TRI_T
        return self.vid(*a) * (3 if d == 1 else 2) + table.index(tuple(corners))

    @staticmethod
    def key(s, order):
        return tuple(sorted((int(order[v]) for v in s), reverse=True))


def canonical_order(f):
    g = np.ascontiguousarray(f, dtype=np.float32).ravel().copy()
    g[g == 0] = 0.0
    idx = np.argsort(g, kind="stable")
    o = np.empty(g.size, dtype=np.int64)
    o[idx] = np.arange(g.size)
    return o


def fields2(rng, shape):
    return [rng.random(shape).astype(np.float32),
            rng.integers(0, 4, size=shape).astype(np.float32),
            rng.choice(np.array([-0.0, 0.0, 1.0, -1.0, np.inf, -np.inf], dtype=np.float32),
                       size=shape)]


def find(parent, a):
    parent.setdefault(a, a)
    while parent[a] != a:
        parent[a] = parent[parent[a]]
        a = parent[a]
    return a


def kruskal_d0(cx, order):
    parent, pairs = {}, []
    for e in sorted(cx.by_dim[1], key=lambda s: cx.key(s, order)):
        a, b = find(parent, e[0]), find(parent, e[1])
        if a == b:
            continue
        if order[a] < order[b]:
            a, b = b, a
        pairs.append((a, e))
        parent[a] = b
    return pairs


def dual_kruskal_d1(cx, order):
    cof = {}
    for t in cx.by_dim[2]:
        for f in itertools.combinations(t, 2):
            cof.setdefault(f, []).append(t)
    parent, pairs = {}, []

    def higher(a, b):
        if a == "OUT":
            return True
        if b == "OUT":
            return False
        return cx.key(a, order) > cx.key(b, order)

    for e in sorted(cx.by_dim[1], key=lambda s: cx.key(s, order), reverse=True):
        ends = cof[e] + ["OUT"] * (2 - len(cof[e]))
        a, b = find(parent, ends[0]), find(parent, ends[1])
        if a == b:
            continue
        if higher(a, b):
            a, b = b, a
        pairs.append((e, a))
        parent[a] = b
    return pairs


def reduction(cx, order):
    allsx = [s for d in range(3) for s in cx.by_dim[d]]
    allsx.sort(key=lambda s: cx.key(s, order))
    pos = {s: i for i, s in enumerate(allsx)}
    pivot, cols, pairs = {}, {}, []
    for j, s in enumerate(allsx):
        col = 0
        if len(s) > 1:
            for f in itertools.combinations(s, len(s) - 1):
                col ^= 1 << pos[f]
        while col and (col.bit_length() - 1) in pivot:
            col ^= cols[pivot[col.bit_length() - 1]]
        if col:
            pivot[col.bit_length() - 1] = j
            cols[j] = col
            pairs.append((allsx[col.bit_length() - 1], s))
    return pairs


def top(s, order):
    return max(s, key=lambda v: order[v])


@pytest.mark.parametrize("shape", [(5, 6), (2, 9), (7, 2), (8, 8)])
def test_order_and_euler(rng, shape):
    for f in fields2(rng, shape):
        r = oracle.run2(f)
        assert np.array_equal(r.order.astype(np.int64), canonical_order(f))
        c = [len(r.crit(d)) for d in range(3)]
        assert c[0] - c[1] + c[2] == 1


@pytest.mark.parametrize("shape", [(5, 6), (4, 9)])
def test_gradient_matching_acyclic_and_lower_link_betti(rng, shape):
    ny, nx = shape
    cx = Complex2(nx, ny)
    ids = {d: {cx.type_id(s): s for s in cx.by_dim[d]} for d in range(3)}
    for f in fields2(rng, shape):
        r = oracle.run2(f)
        order = canonical_order(f)
        gp = r.get(oracle.GRAD_PAIRS2)
        crit = [set(r.crit(d).tolist()) for d in range(3)]
        seen = {d: set() for d in range(3)}
        edges = []  # modified Hasse diagram arcs for the cycle check
        for d, t, h in gp:
            d = int(d)
            ts, hs = ids[d][int(t)], ids[d + 1][int(h)]
            assert set(ts) < set(hs)
            assert top(ts, order) == top(hs, order)
            assert int(t) not in seen[d] and int(h) not in seen[d + 1]
            seen[d].add(int(t))
            seen[d + 1].add(int(h))
            edges.append(((d, int(t)), (d + 1, int(h))))
        for d in range(3):
            assert seen[d].isdisjoint(crit[d])
            assert seen[d] | crit[d] == set(ids[d])
        # acyclic: V-paths alternate up along pairs and down along other facets
        up = {a: b for a, b in edges}
        graph = {}
        for d in (1, 2):
            for i, s in ids[d].items():
                for fct in itertools.combinations(s, len(s) - 1):
                    fi = cx.type_id(fct) if len(fct) > 1 else fct[0]
                    if up.get((d - 1, fi)) != (d, i):
                        graph.setdefault((d, i), []).append((d - 1, fi))
        for a, b in edges:
            graph.setdefault(a, []).append(b)
        state = {}

        def dfs(u):
            state[u] = 1
            for v in graph.get(u, []):
                if state.get(v) == 1:
                    return False
                if v not in state and not dfs(v):
                    return False
            state[u] = 2
            return True
        for u in list(graph):
            if u not in state:
                assert dfs(u)
        # per vertex: critical k-simplices in the lower star = b~_{k-1}(lower link)
        star = {v: {d: [s for s in cx.by_dim[d] if v in s] for d in (1, 2)} for v in range(nx * ny)}
        for v in range(nx * ny):
            low = lambda s: all(order[u] < order[v] for u in s if u != v)
            ledges = [s for s in star[v][1] if low(s)]
            ltris = [s for s in star[v][2] if low(s)]
            lv = [u for s in ledges for u in s if u != v]
            le = [tuple(u for u in s if u != v) for s in ltris]
            if not lv:
                b = (1, 0, 0)
            else:
                parent = {}
                for u in lv:
                    find(parent, u)
                for a, c in le:
                    ra, rc = find(parent, a), find(parent, c)
                    if ra != rc:
                        parent[ra] = rc
                comps = len({find(parent, u) for u in lv})
                b = (0, comps - 1, len(le) - len(lv) + comps)
            got = [0, 0, 0]
            got[0] = int(v in crit[0])
            for e in ledges:
                got[1] += int(cx.type_id(e) in crit[1])
            for t in ltris:
                got[2] += int(cx.type_id(t) in crit[2])
            assert tuple(got) == b, (v, got, b)


@pytest.mark.parametrize("shape", [(5, 6), (3, 8), (7, 7)])
def test_d0_d1_against_kruskal_and_reduction(rng, shape):
    ny, nx = shape
    cx = Complex2(nx, ny)
    for f in fields2(rng, shape):
        r = oracle.run2(f)
        order = canonical_order(f)
        d0 = {(int(p["birth_id"]), int(p["death_id"])) for p in r.get(oracle.D0_2)}
        d1 = {(int(p["birth_id"]), int(p["death_id"])) for p in r.get(oracle.D1_2)}
        k0 = {(m, cx.type_id(e)) for m, e in kruskal_d0(cx, order) if top(e, order) != m}
        k1 = {(cx.type_id(e), cx.type_id(t)) for e, t in dual_kruskal_d1(cx, order)
              if top(e, order) != top(t, order)}
        assert d0 == k0
        assert d1 == k1
        red = reduction(cx, order)
        rd0 = {(b[0], cx.type_id(d)) for b, d in red if len(b) == 1 and top(b, order) != top(d, order)}
        rd1 = {(cx.type_id(b), cx.type_id(d)) for b, d in red
               if len(b) == 2 and top(b, order) != top(d, order)}
        assert d0 == rd0 and d1 == rd1
        ess = r.get(oracle.D0_ESSENTIAL2)
        assert int(ess["birth_id"][0]) == int(np.argmin(order)) and ess["death_id"][0] == -1
        flat = f.ravel()
        for p in list(r.get(oracle.D0_2)) + list(r.get(oracle.D1_2)):
            assert p["birth"] == flat[p["birth_vtx"]] and p["death"] == flat[p["death_vtx"]]
            assert p["death"] >= p["birth"]


@pytest.mark.parametrize("shape", [(4, 5), (9, 3)])
def test_ramp_and_constant_have_one_critical_simplex(shape):
    ny, nx = shape
    for f in (np.arange(nx * ny, dtype=np.float32).reshape(shape),
              np.zeros(shape, dtype=np.float32)):
        r = oracle.run2(f)
        assert [len(r.crit(d)) for d in range(3)] == [1, 0, 0]
        assert len(r.get(oracle.D0_2)) == 0 and len(r.get(oracle.D1_2)) == 0


def test_rejects_nan_and_bad_dims():
    with pytest.raises(oracle.OracleError):
        oracle.run2(np.array([[0, np.nan], [1, 2]], dtype=np.float32))
    with pytest.raises(oracle.OracleError):
        oracle.run2(np.zeros((1, 5), dtype=np.float32))
