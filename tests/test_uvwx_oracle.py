"""Pins of the oracle's parent-neighbour-child lists (U, V, W, X; paper
Section 2.1, after Cheng, Greengard and Rokhlin 1999).

The lists are pinned by what they must do, not by their own formulas:
every directed particle pair is accounted for exactly once (direct, through a
multipole, through a local expansion, or through the particles of an X box),
the potential and its gradient through them tend to the exact direct sum as p
grows, and the
relations between the lists hold (U and V symmetric, X the dual of W, W and X
empty on a tree whose leaves share one level).  A planted slip in any of the
four definitions breaks the coverage."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle import uvwx


def _tree(name, n, leaf):
    wl = W.make_workload(name, n=n)
    return wl, O.build_tree(wl.pos, leaf, 0.5)


@pytest.mark.parametrize("name,n,leaf", [("uniform", 1200, 16), ("plummer", 1200, 8), ("clustered", 1500, 16),
                                         ("clustered", 600, 1)])
def test_every_pair_exactly_once(name, n, leaf):
    _, t = _tree(name, n, leaf)
    lists = uvwx.build_lists(t)
    _, cov = uvwx.coverage(t, lists)
    assert cov.min() == 1 and cov.max() == 1
    bx, U, V, Wl, X = lists
    if name != "uniform":
        assert sum(len(v) for v in Wl.values()) > 0     # the adaptive case is exercised


def test_list_relations():
    _, t = _tree("plummer", 1000, 8)
    bx, U, V, Wl, X = uvwx.build_lists(t)
    for b, us in U.items():
        assert all(b in U[a] for a in us)
    for b, vs in V.items():
        assert all(b in V[c] for c in vs)
        assert all(t.level[c] == t.level[b] for c in vs)
        assert not any(bx.adjacent(b, c) for c in vs)
    for b, ws in Wl.items():
        for d in ws:
            assert b in X[d] and t.level[d] > t.level[b]
            assert not bx.adjacent(b, d) and bx.adjacent(int(t.parent[d]), b)
    assert sum(len(v) for v in Wl.values()) == sum(len(v) for v in X.values())


def test_one_level_tree_has_no_w_or_x():
    """Particles at the centres of a regular 8 x 8 x 8 grid, one per leaf:
    every leaf at level 3, so nothing is finer than a neighbour."""
    g = (np.arange(8) + 0.5) / 8.0
    pos = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    t = O.build_tree(pos, 1, 0.5)
    assert set(t.level[t.is_leaf].tolist()) == {3}
    bx, U, V, Wl, X = uvwx.build_lists(t)
    assert all(len(v) == 0 for v in Wl.values()) and all(len(v) == 0 for v in X.values())
    interior = [b for b in U if np.all(bx.lo[b] > 0) and np.all(bx.hi[b] < (1 << 21))]
    assert interior and all(len(U[b]) == 27 for b in interior)   # the 3 x 3 x 3 block around an inner leaf
    _, cov = uvwx.coverage(t)
    assert cov.min() == 1 and cov.max() == 1


def test_potential_and_field_tend_to_the_direct_sum():
    wl, t = _tree("plummer", 1200, 8)
    lists = uvwx.build_lists(t)
    ref, gref = O.direct(wl.pos, wl.q)
    res = [uvwx.evaluate(wl.pos, wl.q, p, tree=t, lists=lists) for p in (2, 4, 6, 8)]
    err = [O.rel_l2(phi, ref) for phi, _ in res]
    gerr = [O.rel_l2(g, gref) for _, g in res]
    assert all(b < a / 3 for a, b in zip(err, err[1:])), err
    assert all(b < a / 2 for a, b in zip(gerr, gerr[1:])), gerr
    assert err[-1] <= 1e-5 and gerr[-1] <= 1e-4, (err, gerr)


def _mutated(t, which):
    bx, U, V, Wl, X = uvwx.build_lists(t)
    leaves = [c for c in range(t.ncell) if bx.leaf[c]]
    if which == "v_keeps_adjacent":
        for b in range(t.ncell):
            par = int(t.parent[b])
            if par >= 0:
                V[b] = sorted(c for nb in bx.neighbours(par) for c in bx.children[nb] if c != b)
    elif which == "u_same_level_only":
        for b in leaves:
            U[b] = [a for a in U[b] if t.level[a] == t.level[b]]
    elif which == "w_without_parent_test":
        for b in leaves:
            Wl[b] = sorted(d for nb in bx.neighbours(b) for d in bx.descendants(nb) if not bx.adjacent(b, d))
    elif which == "x_missing":
        X = {c: [] for c in range(t.ncell)}
    return bx, U, V, Wl, X


@pytest.mark.parametrize("which", ["v_keeps_adjacent", "u_same_level_only", "w_without_parent_test", "x_missing"])
def test_planted_mistakes_break_coverage(which):
    _, t = _tree("plummer", 800, 8)
    _, cov = uvwx.coverage(t, _mutated(t, which))
    assert cov.min() != 1 or cov.max() != 1


def test_direct_wx_form():
    """W and X as direct sums (the form of the GPU list builder): the P2P pairs
    are symmetric leaf pairs, still cover every particle pair once with V, and
    the result tends to the direct sum like the expansion form."""
    wl, t = _tree("clustered", 1200, 16)
    lists = uvwx.build_lists(t)
    bx, U, V, Wl, X = lists
    m2l, p2p = uvwx.pair_lists(t, lists)
    pairs = set(map(tuple, p2p.tolist()))
    assert all((b, a) in pairs for a, b in pairs)
    assert all(bx.leaf[a] and bx.leaf[b] for a, b in pairs)
    assert len(m2l) == sum(len(v) for v in V.values())
    Ud = {}
    for b, a in p2p:
        Ud.setdefault(int(b), []).append(int(a))
    _, cov = uvwx.coverage(t, (bx, Ud, V, {b: [] for b in Wl}, {c: [] for c in X}))
    assert cov.min() == 1 and cov.max() == 1
    ref, gref = O.direct(wl.pos, wl.q)
    phi, g = uvwx.evaluate(wl.pos, wl.q, 8, tree=t, lists=lists, wx="direct")
    assert O.rel_l2(phi, ref) <= 1e-5 and O.rel_l2(g, gref) <= 1e-4
