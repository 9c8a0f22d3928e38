"""The pairing schedule of the CUDA path, restated step by step in plain
Python on small random extremum graphs and checked against the oracle's
Alg. 1 (``oracle.pair_extrema_saddles``), so that the readings it rests on
are pinned on the CPU and not only through the GPU parity tests:

* Borůvka rounds collect the minimum spanning forest (every component joins
  across its lightest live saddle; a pair of components that chose the same
  saddle hooks one way only), and only the forest's saddles are paired;
* the exact rounds: each root tags its lightest live saddle; a saddle that
  is the lightest of both roots kills the younger (mutual rule), one that
  is the lightest of root a while the other root b is older kills a
  (downhill rule); the rest wait; an immortal node (OUTSIDE) takes no tags;
* the sequential finish in weight order once few saddles are left and the
  rounds stall.

Saddle j is the j-th triplet in visiting order (its weight), ranks are
ages (a larger rank is younger and dies), as in Alg. 1.
"""
import numpy as np
import pytest

import oracle


def _find(parent, x):
    while parent[x] != x:
        parent[x] = parent[parent[x]]
        x = parent[x]
    return x


def _forest(t0, t1, n_nodes, immortal):
    parent = list(range(n_nodes))
    live = [i for i in range(len(t0)) if t0[i] != t1[i]]
    forest = []
    while live:
        roots = {i: (_find(parent, t0[i]), _find(parent, t1[i])) for i in live}
        best = {}
        for i in live:
            for r in roots[i]:
                if roots[i][0] != roots[i][1] and r != immortal:
                    best[r] = min(best.get(r, i), i)
        nxt = []
        for i in live:
            a, b = roots[i]
            if a == b:
                continue
            sa, sb = best.get(a) == i, best.get(b) == i
            if not sa and not sb:
                nxt.append(i)
                continue
            forest.append(i)
            if sa and sb:
                parent[min(a, b)] = max(a, b)
            elif sa:
                parent[a] = b
            else:
                parent[b] = a
        live = nxt
    return forest


def _exact_rounds(live, t0, t1, rank, immortal, seq_max):
    parent = list(range(len(rank)))
    res = [-1] * len(t0)
    prev = None
    while live:
        h = len(live)
        if h <= seq_max and prev is not None and 4 * h > 3 * prev:
            for i in sorted(live):  # the sequential finish, in weight order
                a, b = _find(parent, t0[i]), _find(parent, t1[i])
                if a == b:
                    continue
                young = a if rank[a] > rank[b] else b
                parent[young] = b if young == a else a
                res[i] = young
            break
        prev = h
        roots = {i: (_find(parent, t0[i]), _find(parent, t1[i])) for i in live}
        best = {}
        for i in live:
            a, b = roots[i]
            if a == b:
                continue
            for r in (a, b):
                if r != immortal:
                    best[r] = min(best.get(r, i), i)
        nxt = []
        for i in live:
            a, b = roots[i]
            if a == b:
                continue  # both ends joined: no pair
            la = a != immortal and best.get(a) == i
            lb = b != immortal and best.get(b) == i
            young = None
            if la and lb:
                young = a if rank[a] > rank[b] else b
            elif la and rank[a] > rank[b]:
                young = a
            elif lb and rank[b] > rank[a]:
                young = b
            if young is None:
                nxt.append(i)
            else:
                parent[young] = b if young == a else a
                res[i] = young
        live = nxt
    return res


def schedule(t0, t1, rank, immortal=None, forest_first=True, seq_max=8):
    live = _forest(t0, t1, len(rank), immortal) if forest_first else \
        [i for i in range(len(t0)) if t0[i] != t1[i]]
    return _exact_rounds(sorted(live), t0, t1, rank, immortal, seq_max)


def _random_graph(rng, outside):
    n = int(rng.integers(2, 120))
    m = int(rng.integers(1, 5 * n))
    t0 = rng.integers(0, n, size=m)
    # a few hubs give parallel saddles and long waiting chains
    hubs = rng.integers(0, n, size=3)
    pick = rng.random(m) < 0.3
    t1 = np.where(pick, hubs[rng.integers(0, 3, size=m)], rng.integers(0, n, size=m))
    rank = rng.permutation(n).astype(np.int64)
    if outside:
        rank[0] = -1  # node 0 plays OUTSIDE: older than every extremum
    return [int(x) for x in t0], [int(x) for x in t1], [int(x) for x in rank]


@pytest.mark.parametrize("outside", [False, True])
@pytest.mark.parametrize("forest_first", [True, False])
def test_schedule_equals_alg1(outside, forest_first):
    rng = np.random.default_rng(7 + 2 * outside + forest_first)
    for _ in range(150):
        t0, t1, rank = _random_graph(rng, outside)
        ref = oracle.pair_extrema_saddles(t0, t1, rank)
        for seq_max in (0, 8):
            got = schedule(t0, t1, rank, immortal=0 if outside else None,
                           forest_first=forest_first, seq_max=seq_max)
            assert list(ref) == got


def test_forest_is_kruskal_forest():
    """The Borůvka saddles are exactly the saddles Kruskal keeps."""
    rng = np.random.default_rng(3)
    for _ in range(100):
        t0, t1, rank = _random_graph(rng, False)
        parent = list(range(len(rank)))
        kruskal = []
        for i in range(len(t0)):
            a, b = _find(parent, t0[i]), _find(parent, t1[i])
            if a != b:
                parent[a] = b
                kruskal.append(i)
        assert sorted(_forest(t0, t1, len(rank), None)) == kruskal


def test_schedule_on_the_worked_example():
    """The extremum graph of the paper's self-correcting pairing figure
    (Sec. 4.3, stored under tests/golden with its citation)."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "selfcorrecting_example.json")) as fh:
        g = json.load(fh)
    t = g["triplets"]
    t0 = [x[1] for x in t]
    t1 = [x[2] for x in t]
    rank = list(range(g["n_extrema"]))
    for forest_first in (True, False):
        got = schedule(t0, t1, rank, forest_first=forest_first, seq_max=0)
        assert {(t[j][0], got[j]) for j in range(len(t)) if got[j] >= 0} == \
            {tuple(p) for p in g["pairs"]}


# ------------------------------------------- self-correcting pairing (Alg. 4) --

def _self_correcting(t0, t1, rank, max_rounds=10000):
    """The fixpoint form of the paper's self-correcting pairing (Sec. 4.3,
    Alg. 4) as the GPU runs it: every round every triplet j finds the
    representatives of its ends by following only links assigned by
    earlier triplets (each link records the triplet that assigned it), with
    no path compression; the younger representative is claimed, the earliest
    claimant of an extremum wins, and the winning claims are the next
    round's links.  Returns (per-triplet result, rounds)."""
    n = len(rank)
    link = [None] * n  # (parent, triplet)

    def find(t, j):
        while link[t] is not None and link[t][1] < j:
            t = link[t][0]
        return t

    for rounds in range(1, max_rounds + 1):
        claim = {}
        for j in range(len(t0)):
            a, b = find(t0[j], j), find(t1[j], j)
            if a == b:
                continue
            young, old = (a, b) if rank[a] > rank[b] else (b, a)
            if young not in claim or j < claim[young][1]:
                claim[young] = (old, j)
        nxt = [claim.get(e) for e in range(n)]
        if nxt == link:
            break
        link = nxt
    res = [-1] * len(t0)
    for e in range(n):
        if link[e] is not None:
            res[link[e][1]] = e
    return res, rounds


def test_self_correcting_fixpoint_equals_alg1(rng):
    for _ in range(200):
        n = int(rng.integers(2, 40))
        m = int(rng.integers(1, 90))
        t0 = [int(v) for v in rng.integers(0, n, m)]
        t1 = [int(v) for v in rng.integers(0, n, m)]
        rank = [int(v) for v in rng.permutation(n)]
        res, _ = _self_correcting(t0, t1, rank)
        assert res == [int(v) for v in oracle.pair_extrema_saddles(t0, t1, rank)]


def test_self_correcting_on_chains():
    """Chains of minima: each saddle's representatives come from following
    the earlier saddles' links, so whichever end is older the fixpoint
    settles in a few rounds (where the exact rounds above take one round
    per merge when the minima deepen along the chain)."""
    n = 40
    t0 = list(range(n - 1))
    t1 = list(range(1, n))
    for rank in (list(range(n - 1, -1, -1)), list(range(n))):
        res, rounds = _self_correcting(t0, t1, rank)
        assert res == [int(v) for v in oracle.pair_extrema_saddles(t0, t1, rank)]
        assert rounds <= 3
