"""The v-path walks' path sharing, restated in Python, reaches the ends of
the plain v-paths (Sec. 2.5: the unstable sets of the 1-saddles and the
stable sets of the 2-saddles, the triplets Alg. 1 and its dual pair).

The device walks all saddles at once (paper_2505_21266_gb300/csrc/
dms_pairs.cu, `mark_ends`, `walk_queue`, `link_walks`):

* every end (a minimum for the descending paths, a critical tetrahedron for
  the ascending dual paths) carries an end mark in its claim word before
  the walks start;
* each saddle owns two walks; a walk step claims the current id by a
  compare-and-swap on its claim word: a free word takes the walk's id and
  the walk moves on; a word that holds an end mark ends the walk with that
  end; a word that holds another walk's id ends the walk with a link to
  that walk (from there on both follow the same path);
* a walk leaving the grid (dual paths) ends at OUTSIDE without a claim;
* a walk that ends with a link takes the joined walk's result instead when
  that one is already known (it may itself be a link);
* after all walks, links are followed to an end.

This file runs that protocol on the CPU, with the walks started and
stepped in random interleavings (a bounded number in flight, as in a
persistent grid), on the gradients of small grids from the oracle, and
checks every saddle's two ends against the oracle's triplets.  No GPU is
needed; the GPU tests check the kernels against the oracle."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from refcomplex import Complex

OUTSIDE = -1


def walks(starts, step_to, ends, rng, max_live, eager=True, swap_slots=False):
    """starts[w]: the first id of walk w, or ("end", x) when it has already
    ended (a missing cofacet).  step_to(x): the next id, or OUTSIDE.
    ends: the ids that carry end marks.  Returns the resolved end of every
    walk and the claim words."""
    claim = {x: ("mark", x) for x in ends}
    res = [None] * len(starts)
    pending = list(range(len(starts)))
    rng.shuffle(pending)
    live = {}

    def finish(w, r):
        if eager and r[0] == "link":
            r2 = res[r[1]]
            if r2 is not None:
                r = r2
        res[w] = r

    while pending or live:
        if pending and (not live or (len(live) < max_live and rng.random() < 0.5)):
            w = pending.pop()
            s = starts[w]
            if isinstance(s, tuple):
                finish(w, ("end", s[1]))
            else:
                live[w] = s
            continue
        w = list(live)[rng.integers(len(live))]
        x = live[w]
        old = claim.get(x)
        if old is None:
            claim[x] = ("walk", w)
            nx = step_to(x)
            if nx == OUTSIDE:
                del live[w]
                finish(w, ("end", OUTSIDE))
            else:
                live[w] = nx
        else:
            del live[w]
            finish(w, ("end", old[1]) if old[0] == "mark" else ("link", old[1]))

    def resolve(r):
        for _ in range(len(starts) + 1):
            if r[0] == "end":
                return r[1]
            w = r[1] ^ 1 if swap_slots else r[1]
            r = res[w]
        raise AssertionError("a cycle of links")

    return [resolve(r) for r in res], claim


def _d0_instance(f):
    nz, ny, nx = f.shape
    r = oracle.run(f)
    cx = Complex(nx, ny, nz)
    p0 = r.partner(0)
    minima = set(int(m) for m in r.crit(0))

    def step_to(v):
        code = int(p0[v])
        assert code >= 0 and code & 1, "a vertex on a descending path is paired with an edge"
        a, b = cx.verts(1, code >> 1)
        return b if a == v else a

    starts = []
    for e in r.crit(1):
        a, b = cx.verts(1, int(e))
        starts += [a, b]
    trip = {int(t[0]): {int(t[1]), int(t[2])} for t in r.get(oracle.D0_TRIPLETS)}
    return [int(e) for e in r.crit(1)], starts, step_to, minima, trip


def _d2_instance(f):
    nz, ny, nx = f.shape
    r = oracle.run(f)
    cx = Complex(nx, ny, nz)
    p3 = r.partner(3)
    maxima = set(int(t) for t in r.crit(3))

    cof = {}
    for t in cx.by_dim[3]:
        for tri in cx.facets(t):
            cof.setdefault(cx.id_of(tri), []).append(cx.id_of(t))

    def cofacets(tri):
        return cof.get(tri, [])

    def step_to(t):
        code = int(p3[t])
        assert code >= 0 and not code & 1, "a tet on a dual path is paired with a triangle"
        nxt = [u for u in cofacets(code >> 1) if u != t]
        return nxt[0] if nxt else OUTSIDE

    starts = []
    for s in r.crit(2):
        c2 = cofacets(int(s))
        starts += [c2[0], c2[1] if len(c2) > 1 else ("end", OUTSIDE)]
    trip = {int(t[0]): {int(t[1]), int(t[2])} for t in r.get(oracle.D2_TRIPLETS)}
    return [int(s) for s in r.crit(2)], starts, step_to, maxima, trip


def _fields():
    rng = np.random.default_rng(3)
    yield rng.random((6, 7, 8)).astype(np.float32)
    yield (np.floor(rng.random((7, 6, 6)) * 4) / 4).astype(np.float32)  # ties
    yield rng.random((3, 10, 9)).astype(np.float32)
    z, y, x = np.meshgrid(np.arange(8), np.arange(9), np.arange(7), indexing="ij")
    yield (np.sin(x * 0.9) * np.cos(y * 0.7) + 0.3 * np.sin(z * 1.3)).astype(np.float32)


def _check(saddles, ends, trip):
    for i, s in enumerate(saddles):
        a, b = ends[2 * i], ends[2 * i + 1]
        if s in trip:
            assert {a, b} == trip[s], s
        else:  # both paths end together: no triplet
            assert a == b, s


@pytest.mark.parametrize("k", range(4))
@pytest.mark.parametrize("kind", ["d0", "d2"])
def test_shared_walks_reach_the_oracle_ends(kind, k):
    f = list(_fields())[k]
    saddles, starts, step_to, ends_set, trip = (_d0_instance if kind == "d0" else _d2_instance)(f)
    assert saddles
    for s in range(4):
        rng = np.random.default_rng(100 * k + s)
        max_live = int(rng.choice([1, 3, 32, 10 ** 6]))
        ends, claim = walks(starts, step_to, ends_set, rng, max_live)
        _check(saddles, ends, trip)
        # the end marks are never overwritten
        assert all(claim[x] == ("mark", x) for x in ends_set)


def test_without_eager_results_the_ends_are_the_same():
    f = next(_fields())
    saddles, starts, step_to, ends_set, trip = _d0_instance(f)
    ends, _ = walks(starts, step_to, ends_set, np.random.default_rng(1), 32, eager=False)
    _check(saddles, ends, trip)


def test_a_wrong_result_slot_is_caught():
    """Reading the other walk's slot of a saddle when following a link (a
    plausible slip in the walk-id arithmetic) must fail the checks above:
    wrong ends, or links that never reach an end.  (Without the eager
    results every link is followed at the end, where the slip sits.)"""
    failed = 0
    for k, f in enumerate(_fields()):
        saddles, starts, step_to, ends_set, trip = _d0_instance(f)
        try:
            ends, _ = walks(starts, step_to, ends_set, np.random.default_rng(k), 32,
                            eager=False, swap_slots=True)
            _check(saddles, ends, trip)
        except AssertionError:
            failed += 1
    assert failed == 4
