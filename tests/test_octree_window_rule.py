"""The rule behind the device's one-pass octree, checked on the CPU against the
oracle's recursive tree (Section 2.1: a cell splits while it holds more than
leaf_size particles, down to level 21).

With keys sorted, the level-L cell around particle a is the run of particles
sharing a's level-L prefix, and it holds more than S = leaf_size particles iff
some window of S + 1 consecutive particles containing a shares that prefix.
So a's leaf level is min(1 + max over windows [s, s + S] containing a of the
levels shared by particles s and s + S, 21) (0 when no window exists), and a is
the first particle of the cells of levels (levels shared with a - 1) + 1 up to
its leaf level.  Listing those cells in (level, position) order, with counts,
parents and children found by bisection, must give the oracle's cell table
exactly.  This restates the rule in numpy; it shares nothing with the CUDA
path, and the GPU tests check the kernels against the oracle directly.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

MAXL = 21


def common_levels(k1, k2):
    """Levels two 63-bit Morton keys share (prefixes key >> 3 (21 - L))."""
    x = np.bitwise_xor(k1, k2)
    hb = np.full(x.shape, -1, dtype=np.int64)
    for b in range(63):
        hb = np.where((x >> np.uint64(b)) & np.uint64(1), b, hb)
    return np.where(hb < 0, MAXL, 20 - hb // 3)


def window_max(m, S):
    """out[a] = max(m[s] for s in [a - S, a], s >= 0), by a monotone deque."""
    out = np.empty(len(m), dtype=np.int64)
    dq = []
    for a in range(len(m)):
        while dq and m[dq[-1]] <= m[a]:
            dq.pop()
        dq.append(a)
        if dq[0] < a - S:
            dq.pop(0)
        out[a] = m[dq[0]]
    return out


def octree_by_window_rule(keys, S):
    n = len(keys)
    m = np.full(n, -1, dtype=np.int64)
    if n > S:
        m[: n - S] = common_levels(keys[: n - S], keys[S:])
    M = window_max(m, S)
    hi = np.where(M < 0, 0, np.minimum(M + 1, MAXL))
    lo = np.zeros(n, dtype=np.int64)
    lo[1:] = common_levels(keys[:-1], keys[1:]) + 1
    cells = sorted((L, a) for a in range(n) for L in range(lo[a], hi[a] + 1))
    level = np.array([c[0] for c in cells], dtype=np.int64)
    first = np.array([c[1] for c in cells], dtype=np.int64)
    shift = (3 * (MAXL - level)).astype(np.uint64)
    ckey = keys[first] >> shift
    count = np.empty(len(cells), dtype=np.int64)
    for c, (L, a) in enumerate(cells):
        sh = np.uint64(3 * (MAXL - L))
        count[c] = np.searchsorted(keys >> sh, keys[a] >> sh, side="right") - a
    starts = np.searchsorted(level, np.arange(MAXL + 2))
    parent = np.full(len(cells), -1, dtype=np.int64)
    child_first = np.zeros(len(cells), dtype=np.int64)
    child_count = np.zeros(len(cells), dtype=np.int64)
    for c in range(len(cells)):
        L, a = level[c], first[c]
        if L > 0:
            f = first[starts[L - 1]:starts[L]]
            parent[c] = starts[L - 1] + np.searchsorted(f, a, side="right") - 1
        if count[c] > S and L < MAXL:
            f = first[starts[L + 1]:starts[L + 2]]
            child_first[c] = starts[L + 1] + np.searchsorted(f, a)
            child_count[c] = starts[L + 1] + np.searchsorted(f, a + count[c]) - child_first[c]
    return dict(level=level, cell_key=ckey, first=first, count=count, parent=parent,
                child_first=child_first, child_count=child_count)


def _cases():
    rng = np.random.default_rng(29)
    dup = rng.random((1500, 3))
    dup[300:700] = dup[5]
    line = np.c_[rng.random(1200), np.full(1200, 2.0), np.full(1200, -1.0)]
    return [
        ("uniform S=64", W.make_workload("uniform", n=3000).pos, 64),
        ("plummer S=16", W.make_workload("plummer", n=3000).pos, 16),
        ("clustered S=8", W.make_workload("clustered", n=2500).pos, 8),
        ("plummer S=1", W.make_workload("plummer", n=800).pos, 1),
        ("clustered S=300", W.make_workload("clustered", n=2000).pos, 300),
        ("leaf >= n", rng.random((50, 3)), 50),
        ("coincident", np.tile([[0.25, -3.0, 7.5]], (40, 1)), 4),
        ("duplicates", dup, 8),
        ("line", line, 8),
        ("one", np.array([[0.1, 0.2, 0.3]]), 8),
    ]


@pytest.mark.parametrize("name,pos,S", _cases(), ids=[c[0] for c in _cases()])
def test_window_rule_reproduces_the_oracle_tree(name, pos, S):
    ref = O.build_tree(pos, S, 0.5)
    got = octree_by_window_rule(ref.keys, S)
    assert len(got["level"]) == ref.ncell
    for f in ("level", "cell_key", "first", "count", "parent", "child_first", "child_count"):
        assert np.array_equal(np.asarray(got[f], dtype=np.int64), np.asarray(getattr(ref, f)).astype(np.int64)), f
