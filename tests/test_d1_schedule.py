"""The D1 kernels' round schedule, restated in Python, equals the sequential
homologous propagation (Sec. 2.5 "D1 pairing", Alg. 2 and Alg. 3).

The device runs every column (a critical triangle that D2 left unpaired) at
once, in rounds (paper_2505_21266_gb300/csrc/dms_d1.cu, `advance` and
`publish`):

* a column expands its boundary at the highest edge until that edge is
  critical (an edge paired with a triangle is replaced by the rest of that
  triangle's boundary, Z2);
* it then looks at the owner word of that edge (the smallest key of the
  columns that claimed it): its own key -> stop; larger or unclaimed ->
  claim it by a minimum and stop; smaller -> if that owner settled on the
  edge at the last publish, add the owner's boundary and go on, else wait;
* at the publish step every edge's smallest claimant settles on it.

This file runs that schedule on the CPU, with the columns of a round taken
in a random order and every read of an owner word allowed to see the value
from the start of the round (the device reads it with a plain load while
other columns lower it), and checks that the settled pivots are the pairs of
the sequential reduction: on abstract instances, and on the lower-star
gradients of small grids against the oracle's D1 (itself pinned against a
full boundary-matrix reduction).  No GPU is needed; the GPU tests check the
kernels against the oracle."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from refcomplex import Complex

INF = float("inf")


class Failed(Exception):
    pass


def schedule(cols, rank, boundary, expand, rng, max_rounds=100000):
    """The rounds of `advance` / `publish`.  cols: column ids; rank[c]: the
    column's key (smaller = earlier); boundary[c]: its initial boundary (a
    set, Z2); expand(b): reduces b in place until its highest element is a
    valid pivot and returns it.  Returns {column: pivot} and the number of
    rounds."""
    bnd = {c: set(boundary[c]) for c in cols}
    pivot = {c: None for c in cols}
    settled = {c: False for c in cols}
    owner_key, owner_col = {}, {}
    for rounds in range(1, max_rounds + 1):
        start = dict(owner_key)  # what a plain load may still see this round

        def read(p):
            return (start if rng.random() < 0.5 else owner_key).get(p, INF)

        for c in rng.permutation(len(cols)):
            c = cols[c]
            if settled[c]:
                continue
            while True:
                if pivot[c] is None:
                    pivot[c] = expand(bnd[c])
                p = pivot[c]
                o = read(p)
                if o == rank[c]:
                    break
                if o > rank[c]:
                    owner_key[p] = min(owner_key.get(p, INF), rank[c])
                    break
                oc = owner_col.get(p)
                if oc is None or not settled[oc]:
                    break
                if rank[oc] != o or pivot[oc] != p:
                    break
                bnd[c] ^= bnd[oc]
                pivot[c] = None
        unsettled = 0
        for c in cols:
            own = pivot[c] is not None and owner_key.get(pivot[c]) == rank[c]
            if own:
                owner_col[pivot[c]] = c
            settled[c] = own
            unsettled += not own
        if unsettled == 0:
            return pivot, rounds
    raise Failed("no fixpoint")


def sequential(cols, rank, boundary, expand):
    """Alg. 3's order: columns by increasing key, each reduced by the final
    boundaries of earlier columns until its pivot is unclaimed."""
    owner, fin, out = {}, {}, {}
    for c in sorted(cols, key=lambda c: rank[c]):
        b = set(boundary[c])
        while True:
            p = expand(b)
            if p not in owner:
                break
            b ^= fin[owner[p]]
        owner[p] = c
        fin[c] = b
        out[c] = p
    return out


# ------------------------------------------------------------- abstract --

def _abstract_instance(rng, nrows, ncols):
    """Rows 0..nrows-1 (larger = higher); a random set of them critical;
    every other row r is replaced, when it is the highest, by a random set
    of lower rows (the rest of its paired triangle's boundary)."""
    crit = rng.random(nrows) < 0.45
    subst = {r: set(int(x) for x in rng.choice(r, size=min(r, rng.integers(1, 4)), replace=False))
             for r in range(nrows) if not crit[r]}

    def expand(b):
        while b:
            r = max(b)
            if crit[r]:
                return r
            b ^= {r} | subst[r]
        raise Failed("a column reduced to zero")

    cols = list(range(ncols))
    boundary = {c: set(int(x) for x in rng.choice(nrows, size=rng.integers(2, 6), replace=False))
                for c in cols}
    rank = {c: int(k) for c, k in zip(cols, rng.permutation(ncols))}
    return cols, rank, boundary, expand


def _independent_instance(rng, nrows, ncols):
    """An abstract instance whose columns are independent (none reduces to
    zero, as no D2-unpaired triangle's boundary does), with its sequential
    pivots."""
    while True:
        inst = _abstract_instance(rng, nrows, ncols)
        try:
            return inst, sequential(*inst)
        except Failed:
            continue


@pytest.mark.parametrize("seed", range(40))
def test_rounds_equal_sequential_on_abstract_columns(seed):
    rng = np.random.default_rng(seed)
    nrows = int(rng.integers(30, 90))
    ncols = int(rng.integers(5, 25))
    (cols, rank, boundary, expand), ref = _independent_instance(rng, nrows, ncols)
    got, rounds = schedule(cols, rank, boundary, expand, rng)
    assert got == ref
    # the earliest column not yet in its final state settles every round
    assert rounds <= ncols + 1


def test_stale_reads_and_orders_do_not_change_the_pivots():
    """The same instance under many schedules (orders, stale reads)."""
    (cols, rank, boundary, expand), ref = _independent_instance(np.random.default_rng(123), 80, 30)
    for s in range(25):
        got, _ = schedule(cols, rank, boundary, expand, np.random.default_rng(s))
        assert got == ref


# ----------------------------------------------------- lower-star gradient --

def _grid_instance(f):
    """Columns, keys, boundaries and the expansion of the D1 kernels, built
    from the oracle's gradient and D0 / D2 pairs of the field f."""
    nz, ny, nx = f.shape
    r = oracle.run(f, d1=True)
    order = r.order
    cx = Complex(nx, ny, nz)
    p1 = r.partner(1)
    crit1 = set(int(e) for e in r.crit(1))
    d0_dead = set(int(e) for e in r.get(oracle.D0)["death_id"])
    d2_born = set(int(t) for t in r.get(oracle.D2)["birth_id"])

    def edges_of(t):
        return {cx.id_of(e) for e in cx.facets(cx.verts(2, t))}

    ekey = {e: cx.key(cx.verts(1, e), order) for e in (cx.id_of(s) for s in cx.by_dim[1])}

    def expand(b):
        while b:
            e = max(b, key=lambda x: ekey[x])
            if e in crit1:
                if e in d0_dead:
                    raise Failed("a D0 edge as the highest edge of a cycle")
                return e
            code = int(p1[e])
            if code < 0 or not code & 1:
                raise Failed("an edge paired with a vertex as the highest edge of a cycle")
            b ^= edges_of(code >> 1)  # the paired triangle's boundary: e cancels
        raise Failed("a column reduced to zero")

    cols = sorted(int(t) for t in r.crit(2) if int(t) not in d2_born)
    tkey = {t: cx.key(cx.verts(2, t), order) for t in cols}
    ranked = sorted(cols, key=lambda t: tkey[t])
    rank = {t: i for i, t in enumerate(ranked)}
    boundary = {t: edges_of(t) for t in cols}
    pairs = {(int(p["birth_id"]), int(p["death_id"])) for p in r.get(oracle.D1)}
    return cols, rank, boundary, expand, pairs


def _fields():
    rng = np.random.default_rng(7)
    yield rng.random((5, 6, 7)).astype(np.float32)
    yield (np.floor(rng.random((6, 6, 6)) * 4) / 4).astype(np.float32)  # ties
    yield rng.random((3, 9, 8)).astype(np.float32)
    yield (np.floor(rng.random((7, 5, 6)) * 16) / 16).astype(np.float32)
    yield rng.random((10, 11, 12)).astype(np.float32)  # ~200 columns, 5+ rounds
    yield (np.floor(rng.random((12, 10, 9)) * 8) / 8).astype(np.float32)


@pytest.mark.parametrize("k", range(6))
def test_rounds_on_lower_star_gradients_give_the_oracle_d1(k):
    f = list(_fields())[k]
    cols, rank, boundary, expand, pairs = _grid_instance(f)
    assert cols, "the field has D1 pairs"
    ref = sequential(cols, rank, boundary, expand)
    assert {(e, t) for t, e in ref.items()} == pairs
    for s in range(3):
        got, rounds = schedule(cols, rank, boundary, expand, np.random.default_rng(s))
        assert {(e, t) for t, e in got.items()} == pairs
        assert rounds <= len(cols) + 1


def test_a_reversed_claim_is_caught():
    """The earliest claimant of an edge must win (a minimum over column
    keys): with the comparison reversed (a maximum, the latest column wins)
    earlier columns add later ones and the pivots are no longer Alg. 3's,
    so the tests above would see that mistake.  (Which settled owner's
    boundary is added does not change the pivots in this sequential model:
    every addition is of an earlier column; the settled check guards the
    device against reading a boundary while its column rewrites it.)"""
    differs = 0
    for seed in range(10):
        rng = np.random.default_rng(seed)
        (cols, rank, boundary, expand), ref = _independent_instance(rng, 60, 25)
        got, _ = schedule(cols, {c: -rank[c] for c in cols}, boundary, expand, rng)
        differs += got != ref
    assert differs > 0
