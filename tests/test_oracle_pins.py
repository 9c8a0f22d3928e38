"""Pins of the CPU oracle against what the paper and the mathematics fix.

Every check below compares the oracle with something other than itself:
numpy's stable argsort (order), the definition of a discrete gradient field
(valid matching, shared maximum vertex, no closed v-path), Robins et al.'s
guarantee that the critical cells of a lower star count the reduced homology
of the lower link (Sec. 2.3), the Euler characteristic of the grid, union-find
over ALL edges / all tetrahedra (the elder rule of Sec. 2.4 applied to the
whole lexicographic filtration), a full Z2 boundary-matrix reduction, and the
worked example of the self-correcting-pairing figure (Sec. 4.3).
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
import refcomplex as rc

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def fields(rng, shape, kinds=("uniform", "ties", "signed_zero")):
    out = []
    for k in kinds:
        if k == "uniform":
            out.append(rng.random(shape).astype(np.float32))
        elif k == "ties":
            out.append(rng.integers(0, 4, size=shape).astype(np.float32))
        elif k == "signed_zero":
            f = rng.choice(np.array([-0.0, 0.0, 1.0, -1.0, np.inf, -np.inf], dtype=np.float32),
                           size=shape)
            out.append(f.astype(np.float32))
    return out


# ----------------------------------------------------------------- order ----

@pytest.mark.parametrize("shape", [(2, 2, 2), (3, 5, 4), (7, 6, 9)])
def test_order_is_stable_argsort(rng, shape):
    for f in fields(rng, shape):
        r = oracle.run(f, gradient=False, diagrams=False)
        assert np.array_equal(r.order.astype(np.int64), rc.canonical_order(f))


def test_order_rejects_nan_and_bad_dims():
    f = np.zeros((3, 3, 3), np.float32)
    f[1, 1, 1] = np.nan
    with pytest.raises(oracle.OracleError):
        oracle.run(f)
    with pytest.raises(oracle.OracleError):
        oracle.run(np.zeros((1, 3, 3), np.float32))


# -------------------------------------------------------------- gradient ----

def _check_gradient(f, r, cx):
    order = rc.canonical_order(f)
    part = [r.partner(d) for d in range(4)]
    for d in range(4):
        # every existing simplex is critical or paired; absent ids are absent
        ex = np.array([cx.exists(d, i) for i in range(len(part[d]))])
        assert np.all((part[d] == oracle.ABSENT) == ~ex)
        for i in np.nonzero(ex)[0]:
            p = int(part[d][i])
            if p == oracle.CRITICAL:
                continue
            up, j = p & 1, p >> 1
            e = d + 1 if up else d - 1
            assert 0 <= e <= 3
            back = int(part[e][j])
            assert back >= 0 and (back >> 1) == i and (back & 1) == (0 if up else 1)
            tail, head = (cx.verts(d, i), cx.verts(e, j)) if up else (cx.verts(e, j), cx.verts(d, i))
            assert set(tail) < set(head) and len(head) == len(tail) + 1
            # both simplices lie in the lower star of the same vertex
            assert cx.max_vertex(tail, order) == cx.max_vertex(head, order)
    return part, order


def _check_acyclic(cx, part):
    """No closed v-path: for each d, the graph tail -> other facets of head
    must be acyclic (Sec. 2.3, definition of a discrete gradient field)."""
    for d in range(3):
        succ = {}
        for i, p in enumerate(part[d]):
            if p >= 0 and (p & 1):
                head = cx.verts(d + 1, int(p >> 1))
                tail = cx.verts(d, i)
                succ[tail] = [f for f in cx.facets(head) if f != tail]
        state = {}
        for s0 in succ:
            if s0 in state:
                continue
            stack = [(s0, iter(succ.get(s0, [])))]
            state[s0] = 1
            while stack:
                node, it = stack[-1]
                nxt = next(it, None)
                if nxt is None:
                    state[node] = 2
                    stack.pop()
                    continue
                st = state.get(nxt, 0)
                assert st != 1, f"closed v-path through {nxt} (dim {d})"
                if st == 0:
                    state[nxt] = 1
                    stack.append((nxt, iter(succ.get(nxt, []))))


@pytest.mark.parametrize("shape", [(2, 2, 2), (4, 3, 5), (6, 6, 6)])
def test_gradient_is_acyclic_matching(rng, shape):
    for f in fields(rng, shape):
        r = oracle.run(f, diagrams=False)
        cx = rc.Complex(shape[2], shape[1], shape[0])
        part, _ = _check_gradient(f, r, cx)
        _check_acyclic(cx, part)


@pytest.mark.parametrize("shape", [(5, 4, 6), (6, 6, 6)])
def test_critical_counts_are_lower_link_betti(rng, shape):
    """Robins et al. (Sec. 2.3): in 3D the critical k-cells in the lower star
    of x are as many as the reduced (k-1)-Betti number of its lower link."""
    for f in fields(rng, shape):
        r = oracle.run(f, diagrams=False)
        cx = rc.Complex(shape[2], shape[1], shape[0])
        order = rc.canonical_order(f)
        star = {v: {d: [] for d in (1, 2, 3)} for v in range(cx.n)}
        for d in (1, 2, 3):
            for s in cx.by_dim[d]:
                for v in s:
                    star[v][d].append(s)
        counts = np.zeros((cx.n, 4), dtype=np.int64)
        for d in range(4):
            for i in r.crit(d):
                counts[cx.max_vertex(cx.verts(d, int(i)), order), d] += 1
        for v in range(cx.n):
            assert tuple(counts[v]) == rc.lower_link_reduced_betti(cx, order, v, star[v]), v


@pytest.mark.parametrize("shape", [(3, 3, 3), (9, 7, 8), (16, 16, 16)])
def test_euler_characteristic(rng, shape):
    for f in fields(rng, shape):
        r = oracle.run(f, diagrams=False)
        c = [len(r.crit(d)) for d in range(4)]
        assert c[0] - c[1] + c[2] - c[3] == 1


def test_critical_lists_are_the_unpaired_simplices(rng):
    f = rng.random((5, 6, 7)).astype(np.float32)
    r = oracle.run(f, diagrams=False)
    for d in range(4):
        p = r.partner(d)
        assert np.array_equal(r.crit(d), np.nonzero(p == oracle.CRITICAL)[0])


# -------------------------------------------------------------- diagrams ----

def _d0_set(r):
    return {(int(p["birth_id"]), int(p["death_id"])) for p in r.get(oracle.D0)}


def _d2_set(r):
    return {(int(p["birth_id"]), int(p["death_id"])) for p in r.get(oracle.D2)}


@pytest.mark.parametrize("shape", [(3, 4, 5), (7, 7, 7), (10, 9, 8)])
def test_d0_equals_kruskal_over_all_edges(rng, shape):
    """The DMS D0 pairs are the elder-rule pairs of ALL edges in
    lexicographic order whose dying vertex is not the edge's own top vertex;
    those that are, are exactly the gradient's vertex-edge pairs."""
    for f in fields(rng, shape):
        r = oracle.run(f)
        cx = rc.Complex(shape[2], shape[1], shape[0])
        order = rc.canonical_order(f)
        kr = rc.kruskal_d0(cx, order)
        nonzero = {(v, cx.id_of(e)) for v, e in kr if cx.max_vertex(e, order) != v}
        zero = {(v, cx.id_of(e)) for v, e in kr if cx.max_vertex(e, order) == v}
        assert _d0_set(r) == nonzero
        gp = r.get(oracle.GRAD_PAIRS)
        ve = {(int(t), int(h)) for d, t, h in gp if d == 0}
        assert ve == zero
        ess = r.get(oracle.D0_ESSENTIAL)
        assert len(ess) == 1 and int(ess[0]["birth_id"]) == int(np.argmin(order))
        assert len(r.get(oracle.D0)) == len(r.crit(0)) - 1


@pytest.mark.parametrize("shape", [(3, 4, 5), (7, 7, 7), (9, 8, 10)])
def test_d2_equals_dual_kruskal(rng, shape):
    """The DMS D2 pairs are the elder-rule pairs of the dual graph
    (tetrahedra + outside, triangles in decreasing order) between simplices
    with different top vertices."""
    for f in fields(rng, shape):
        r = oracle.run(f)
        cx = rc.Complex(shape[2], shape[1], shape[0])
        order = rc.canonical_order(f)
        dk = rc.dual_kruskal_d2(cx, order)
        nonzero = {(cx.id_of(s), cx.id_of(t)) for s, t in dk
                   if cx.max_vertex(s, order) != cx.max_vertex(t, order)}
        zero = {(cx.id_of(s), cx.id_of(t)) for s, t in dk
                if cx.max_vertex(s, order) == cx.max_vertex(t, order)}
        assert _d2_set(r) == nonzero
        # the tetrahedra outside the zero-persistence dual pairs are the
        # critical ones (the zero-persistence skip of Sec. 2.5)
        tets = {int(i) for i in range(len(r.partner(3))) if r.partner(3)[i] != oracle.ABSENT}
        assert tets - {t for _, t in zero} == set(int(i) for i in r.crit(3))
        assert len(r.get(oracle.D2)) == len(r.crit(3))


@pytest.mark.parametrize("shape", [(2, 2, 2), (4, 3, 5), (5, 5, 5)])
def test_all_pairs_equal_boundary_matrix_reduction(rng, shape):
    """Full Z2 reduction of the lexicographic filtration: its pairs between
    simplices of different top vertices are the D0/D2 pairs (plus D1), its
    zero-persistence pairs are the gradient pairs (the zero-persistence skip
    of Sec. 2.5), its essential classes are the global minimum alone."""
    for f in fields(rng, shape):
        r = oracle.run(f, reduction=True)
        cx = rc.Complex(shape[2], shape[1], shape[0])
        order = rc.canonical_order(f)
        pairs, ess = rc.reduction_pairs(cx, order)
        top = lambda s: cx.max_vertex(s, order)
        d0 = {(b[0], cx.id_of(dd)) for b, dd in pairs if len(b) == 1 and top(b) != top(dd)}
        d2 = {(cx.id_of(b), cx.id_of(dd)) for b, dd in pairs if len(b) == 3 and top(b) != top(dd)}
        assert _d0_set(r) == d0
        assert _d2_set(r) == d2
        zero = {(len(b) - 1, cx.id_of(b), cx.id_of(dd)) for b, dd in pairs if top(b) == top(dd)}
        gp = {tuple(int(x) for x in row) for row in r.get(oracle.GRAD_PAIRS)}
        # vertex-edge gradient pairs are exactly the zero-persistence pairs of
        # dimension 0; in dimensions 1 and 2 the gradient may pick another
        # zero-persistence partner, but it leaves exactly the same simplices
        # critical (Sec. 2.5, zero-persistence skip)
        assert {p for p in gp if p[0] == 0} == {p for p in zero if p[0] == 0}
        in_zero = {(d, i) for d, i, _ in zero} | {(d + 1, j) for d, _, j in zero}
        crit = {(d, int(i)) for d in range(4) for i in r.crit(d)}
        every = {(d, cx.id_of(s)) for d in range(4) for s in cx.by_dim[d]}
        assert every - in_zero == crit
        # the remaining (D1) pairs join critical edges to critical triangles
        for b, dd in pairs:
            if top(b) != top(dd):
                assert (len(b) - 1, cx.id_of(b)) in crit and (len(dd) - 1, cx.id_of(dd)) in crit
        assert [len(s) for s in ess] == [1] and ess[0][0] == int(np.argmin(order))
        # the oracle's own reduction agrees with this one
        red = r.get(oracle.REDUCTION)
        mine = {(len(b) - 1, cx.id_of(b), cx.id_of(dd)) for b, dd in pairs}
        mine |= {(len(s) - 1, cx.id_of(s), -1) for s in ess}
        assert {tuple(int(x) for x in row) for row in red} == mine


def test_two_by_two_by_two_all_orders_sampled(rng):
    """The 2x2x2 grid (one cube, 6 tets): random permutations of the 8
    vertex values against the full reduction."""
    cx = rc.Complex(2, 2, 2)
    for _ in range(300):
        f = rng.permutation(8).astype(np.float32).reshape(2, 2, 2)
        r = oracle.run(f)
        order = rc.canonical_order(f)
        pairs, _ = rc.reduction_pairs(cx, order)
        top = lambda s: cx.max_vertex(s, order)
        zero = {(len(b) - 1, cx.id_of(b), cx.id_of(dd)) for b, dd in pairs if top(b) == top(dd)}
        gp = {tuple(int(x) for x in row) for row in r.get(oracle.GRAD_PAIRS)}
        assert {p for p in gp if p[0] == 0} == {p for p in zero if p[0] == 0}
        in_zero = {(d, i) for d, i, _ in zero} | {(d + 1, j) for d, _, j in zero}
        crit = {(d, int(i)) for d in range(4) for i in r.crit(d)}
        every = {(d, cx.id_of(s)) for d in range(4) for s in cx.by_dim[d]}
        assert every - in_zero == crit
        d0 = {(b[0], cx.id_of(dd)) for b, dd in pairs if len(b) == 1 and top(b) != top(dd)}
        assert _d0_set(r) == d0


def test_values_are_copies_of_input_floats(rng):
    f = rng.random((8, 9, 10)).astype(np.float32)
    r = oracle.run(f)
    flat = f.ravel()
    order = rc.canonical_order(f)
    for name in (oracle.D0, oracle.D2):
        for p in r.get(name):
            assert p["birth"] == flat[p["birth_vtx"]] and p["death"] == flat[p["death_vtx"]]
            assert p["death"] >= p["birth"]
            assert order[p["death_vtx"]] > order[p["birth_vtx"]]


# --------------------------------------------------------- special cases ----

@pytest.mark.parametrize("shape", [(2, 2, 2), (5, 4, 3), (12, 11, 10)])
def test_ramp_and_constant_have_one_critical_simplex(shape):
    """f = vertex offset, and a constant field (all ties fall to the offset):
    one minimum, no other critical simplex, empty D0/D2 (the "Elevation"
    shape of Sec. 6.1)."""
    n = int(np.prod(shape))
    for f in (np.arange(n, dtype=np.float32).reshape(shape), np.full(shape, 3.5, np.float32)):
        r = oracle.run(f)
        assert [len(r.crit(d)) for d in range(4)] == [1, 0, 0, 0]
        assert r.crit(0)[0] == 0
        assert len(r.get(oracle.D0)) == 0 and len(r.get(oracle.D2)) == 0


# --------------------------------------------------- worked example (Alg.1) --

def test_self_correcting_figure_example():
    with open(os.path.join(GOLDEN, "selfcorrecting_example.json")) as fh:
        g = json.load(fh)
    t = np.array(g["triplets"], dtype=np.int64)
    res = oracle.pair_extrema_saddles(t[:, 1], t[:, 2], np.arange(g["n_extrema"]))
    got = {(int(t[j, 0]), int(res[j])) for j in range(len(t)) if res[j] >= 0}
    assert got == {tuple(p) for p in g["pairs"]}
    paired = {p for _, p in got}
    assert [e for e in range(g["n_extrema"]) if e not in paired] == g["essential"]


def test_pair_extrema_saddles_matches_kruskal_on_random_graphs(rng):
    """Alg. 1 on random extremum graphs equals union-find with the elder
    rule written independently (Sec. 2.5)."""
    for _ in range(50):
        n = int(rng.integers(2, 30))
        m = int(rng.integers(1, 60))
        t0 = rng.integers(0, n, m)
        t1 = rng.integers(0, n, m)
        keep = t0 != t1
        t0, t1 = t0[keep], t1[keep]
        rank = rng.permutation(n)
        res = oracle.pair_extrema_saddles(t0, t1, rank)
        parent = list(range(n))

        def find(a):
            while parent[a] != a:
                a = parent[a]
            return a
        for j in range(len(t0)):
            a, b = find(t0[j]), find(t1[j])
            if a == b:
                assert res[j] == -1
                continue
            young, old = (a, b) if rank[a] > rank[b] else (b, a)
            assert res[j] == young
            parent[young] = old


# ------------------------------------------------ sampled lower stars ----

def test_lower_star_vertex_from_field_matches_full_gradient(rng):
    f = rng.integers(0, 6, size=(6, 7, 8)).astype(np.float32)
    r = oracle.run(f, diagrams=False)
    gp = {tuple(int(x) for x in row) for row in r.get(oracle.GRAD_PAIRS)}
    crit = {(d, int(i)) for d in range(4) for i in r.crit(d)}
    cx = rc.Complex(8, 7, 6)
    order = rc.canonical_order(f)
    for v in range(cx.n):
        pairs, cr = oracle.lower_star_vertex(f, v)
        mine_p = {tuple(int(x) for x in row) for row in pairs}
        mine_c = {(int(d), int(i)) for d, i in cr}
        exp_p = {p for p in gp if cx.max_vertex(cx.verts(p[0], p[1]), order) == v}
        exp_c = {c for c in crit if cx.max_vertex(cx.verts(*c), order) == v}
        assert mine_p == exp_p and mine_c == exp_c


@pytest.mark.parametrize("shape", [(5, 6, 7), (4, 4, 9), (2, 3, 11)])
def test_local_elder_rule_matches_full_diagrams(rng, shape):
    """The local checks (components grown from the two ends of one simplex)
    agree with the full D0 / D2 on every critical edge and triangle: they
    report a death exactly for the pairs the diagrams hold, with the same
    dying extremum; and every gradient vertex-edge pair is a zero-persistence
    death of its top vertex."""
    for f in fields(rng, shape):
        r = oracle.run(f)
        d0 = {int(p["death_id"]): int(p["birth_id"]) for p in r.get(oracle.D0)}
        for e in r.crit(1):
            st, dying = oracle.d0_edge_local(f, int(e))
            if int(e) in d0:
                assert st == 1 and dying == d0[int(e)]
            else:
                assert st == 0
        d2 = {int(p["birth_id"]): int(p["death_id"]) for p in r.get(oracle.D2)}
        for t in r.crit(2):
            st, dying = oracle.d2_triangle_local(f, int(t))
            if int(t) in d2:
                assert st == 1 and dying == d2[int(t)]
            else:
                assert st == 0
        gp = r.get(oracle.GRAD_PAIRS).reshape(-1, 3)
        for dim, v, e in gp[gp[:, 0] == 0][:40]:
            assert oracle.d0_edge_local(f, int(e)) == (1, int(v))


def test_local_elder_rule_limit(rng):
    f = rng.random((12, 12, 12)).astype(np.float32)
    r = oracle.run(f, gradient=True, diagrams=False)
    outcomes = {oracle.d0_edge_local(f, int(e), limit=3)[0] for e in r.crit(1)}
    assert -1 in outcomes


def _bottleneck(a, b):
    """Bottleneck distance between two finite diagrams (arrays [n, 2]) under
    the L-infinity norm, points free to match the diagonal: the smallest
    candidate threshold at which the usual bipartite graph (points of a and
    diagonal copies of b's points against points of b and diagonal copies of
    a's) has a perfect matching."""
    nx_ = pytest.importorskip("networkx")
    a = np.asarray(a, dtype=np.float64).reshape(-1, 2)
    b = np.asarray(b, dtype=np.float64).reshape(-1, 2)
    da, db = (a[:, 1] - a[:, 0]) / 2, (b[:, 1] - b[:, 0]) / 2
    cand = {0.0, *da.tolist(), *db.tolist()}
    for p in a:
        for q in b:
            cand.add(float(np.max(np.abs(p - q))))
    for t in sorted(cand):
        g = nx_.Graph()
        left = [("a", i) for i in range(len(a))] + [("da", j) for j in range(len(b))]
        right = [("b", j) for j in range(len(b))] + [("db", i) for i in range(len(a))]
        g.add_nodes_from(left, bipartite=0)
        g.add_nodes_from(right, bipartite=1)
        for i in range(len(a)):
            for j in range(len(b)):
                if np.max(np.abs(a[i] - b[j])) <= t:
                    g.add_edge(("a", i), ("b", j))
            if da[i] <= t:
                g.add_edge(("a", i), ("db", i))
        for j in range(len(b)):
            if db[j] <= t:
                g.add_edge(("da", j), ("b", j))
        for j in range(len(b)):
            for i in range(len(a)):
                g.add_edge(("da", j), ("db", i))
        m = nx_.bipartite.hopcroft_karp_matching(g, top_nodes=left)
        if len(m) // 2 == len(left):
            return t
    return float("inf")


def test_bottleneck_helper_on_hand_diagrams():
    assert _bottleneck([[0, 1]], [[0, 1]]) == 0
    assert _bottleneck([[0, 1]], [[0.1, 1.2]]) == pytest.approx(0.2)
    assert _bottleneck([[0, 1]], []) == pytest.approx(0.5)  # to the diagonal
    assert _bottleneck([[0, 4], [1, 1.2]], [[0.5, 4]]) == pytest.approx(0.5)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_diagrams_are_stable_under_perturbation(seed):
    """Stability of persistence diagrams: the bottleneck distance between the
    D0 (and D2) value diagrams of f and f + e is at most max |e|, and the
    essential minimum moves by at most max |e| too."""
    rng = np.random.default_rng(100 + seed)
    f = rng.random((5, 6, 7)).astype(np.float32)
    e = ((rng.random(f.shape) - 0.5) * 0.02).astype(np.float32)
    g = (f + e).astype(np.float32)
    eps = float(np.max(np.abs(g.astype(np.float64) - f.astype(np.float64))))
    rf, rg = oracle.run(f), oracle.run(g)
    for which in (oracle.D0, oracle.D2):
        pf, pg = rf.get(which), rg.get(which)
        a = np.stack([pf["birth"], pf["death"]], 1)
        b = np.stack([pg["birth"], pg["death"]], 1)
        assert _bottleneck(a, b) <= eps + 1e-9
    ef, eg = rf.get(oracle.D0_ESSENTIAL), rg.get(oracle.D0_ESSENTIAL)
    assert abs(float(ef["birth"][0]) - float(eg["birth"][0])) <= eps + 1e-9


# ------------------------------- hand-worked lower stars (Sec. 2.3) --------

_NEIGHBOUR_OFFSETS = {
    "X+": (1, 0, 0), "X-": (-1, 0, 0), "Y+": (0, 1, 0), "Y-": (0, -1, 0),
    "Z+": (0, 0, 1), "Z-": (0, 0, -1), "XY+": (1, 1, 0), "XY-": (-1, -1, 0),
    "XZ+": (1, 0, 1), "XZ-": (-1, 0, -1), "YZ+": (0, 1, 1), "YZ-": (0, -1, -1),
    "D+": (1, 1, 1), "D-": (-1, -1, -1)}


def golden_lower_stars():
    """The cases of tests/golden/lower_stars.json as (name, field, expected
    pairs as (tail_dim, tail_id, head_id), expected criticals as (dim, id))
    on a 3x3x3 grid whose centre vertex is x; ids from refcomplex's own
    restatement of the documented id convention."""
    with open(os.path.join(GOLDEN, "lower_stars.json")) as fh:
        g = json.load(fh)
    cx = rc.Complex(3, 3, 3)
    x = cx.vid(1, 1, 1)

    def vertex(label):
        if label == "x":
            return x
        dx, dy, dz = _NEIGHBOUR_OFFSETS[label]
        return cx.vid(1 + dx, 1 + dy, 1 + dz)

    def simplex(text):
        s = tuple(sorted(vertex(t) for t in text.split()))
        return len(s) - 1, cx.type_id(s)

    out = []
    for case in g["cases"]:
        f = 100.0 + np.arange(27, dtype=np.float32)
        f[x] = 50.0
        for label, r in case["lower"].items():
            f[vertex(label)] = 1.0 + r
        pairs = set()
        for tail, head in case["pairs"]:
            (dt, it), (_, ih) = simplex(tail), simplex(head)
            pairs.add((dt, it, ih))
        crit = {simplex(t) for t in case["critical"]}
        out.append((case["name"], f.reshape(3, 3, 3), x, pairs, crit))
    return out


@pytest.mark.parametrize("case", golden_lower_stars(), ids=lambda c: c[0])
def test_lower_star_partners_match_hand_worked_cases(case):
    """Which edge pairs with which triangle and which triangle with which tet
    (the choice ProcessLowerStars makes, not only the critical counts),
    against lower stars worked by hand from the algorithm's steps."""
    name, f, x, exp_pairs, exp_crit = case
    pairs, crit = oracle.lower_star_vertex(f, x)
    assert {tuple(int(v) for v in row) for row in pairs} == exp_pairs, name
    assert {(int(d), int(i)) for d, i in crit} == exp_crit, name
    # the whole-grid run agrees on the lower star of x
    r = oracle.run(f, diagrams=False)
    cx = rc.Complex(3, 3, 3)
    order = rc.canonical_order(f)
    gp = {tuple(int(v) for v in row) for row in r.get(oracle.GRAD_PAIRS)
          if cx.max_vertex(cx.verts(int(row[0]), int(row[1])), order) == x}
    assert gp == exp_pairs, name


def test_threaded_gradient_equals_single_threaded(rng):
    """The CPU baseline's shape -- the lower stars of z-slabs on several host
    threads -- gives the oracle's single-threaded result exactly."""
    f = rng.integers(0, 7, size=(9, 8, 10)).astype(np.float32)
    a = oracle.run(f)
    b = oracle.run(f, threads=4)
    for w in (oracle.GRAD_PAIRS, oracle.CRIT0, oracle.CRIT1, oracle.CRIT2, oracle.CRIT3):
        assert np.array_equal(a.get(w), b.get(w))
    for w in (oracle.D0, oracle.D2):
        assert a.get(w).tobytes() == b.get(w).tobytes()


# ------------------------------------------------------------ D1 (Alg. 2-3) --

@pytest.mark.parametrize("shape", [(2, 2, 2), (4, 5, 3), (7, 6, 8), (12, 12, 12)])
def test_d1_equals_boundary_matrix_reduction(rng, shape):
    """The oracle's D1 (homologous propagation over the critical triangles
    D2 left unpaired, Sec. 2.5, Alg. 2-3) equals the (edge, triangle) pairs
    of a full Z2 reduction of the lexicographic filtration whose two
    simplices have different highest vertices, id for id; and every
    critical edge / triangle is in exactly one of D0, D1 / D1, D2."""
    nz, ny, nx = shape
    cx = rc.Complex(nx, ny, nz)
    for f in fields(rng, shape) + [rc_mixture(shape)]:
        r = oracle.run(f, d1=True, reduction=True)
        order = rc.canonical_order(f)
        exp = {(int(b), int(d)) for dim, b, d in r.get(oracle.REDUCTION)
               if dim == 1 and d >= 0
               and cx.max_vertex(cx.verts(1, int(b)), order) != cx.max_vertex(cx.verts(2, int(d)), order)}
        d1 = r.get(oracle.D1)
        assert {(int(p["birth_id"]), int(p["death_id"])) for p in d1} == exp
        assert len(d1) == len(r.crit(1)) - len(r.get(oracle.D0)) == len(r.crit(2)) - len(r.get(oracle.D2))
        fl = f.ravel()
        assert np.array_equal(d1["birth"].view(np.uint32), fl[d1["birth_vtx"]].view(np.uint32))
        assert np.array_equal(d1["death"].view(np.uint32), fl[d1["death_vtx"]].view(np.uint32))


def rc_mixture(shape):
    from paper_2505_21266_gb300 import fields as F
    return F.gaussian_mixture(shape, 4, (0.1, 0.3), 1e-3, 5).numpy()
