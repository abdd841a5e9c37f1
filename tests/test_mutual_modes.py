"""The record-mode rule of the mutual near field (paper Section 4: one
evaluation of a pair serves both cells), checked on the host.

Every P2P record (target a, source b) gets a mode from one question, "is a in
b's list" (y):  b == a -> 0;  b > a -> 2 if y else 1;  b < a -> 0 if y else 1.
Mode 2 evaluates both directions, mode 1 only a <- b, mode 0 nothing (the own
pairs go to the own-leaf kernel).  The rule must evaluate every directed
cross-leaf pair of the lists exactly once for any lists, symmetric or not; the
dual traversal's lists are symmetric on the workload recipes (so on the GPU
every cross-leaf record has mode 2 or 0), which the second test pins on the
oracle's trees."""
import numpy as np
import pytest

import oracle as O
import workloads as W


def modes(records):
    """The rule, written from its statement above (records: (a, b) pairs)."""
    present = set(map(tuple, records))
    out = []
    for a, b in records:
        if a == b:
            out.append(0)
            continue
        y = (b, a) in present
        out.append((2 if y else 1) if b > a else (0 if y else 1))
    return out


def evaluated(records):
    """Directed pairs (target, source) each mode evaluates, with multiplicity."""
    got = {}
    for (a, b), m in zip(map(tuple, records), modes(records)):
        for d in ([(a, b), (b, a)] if m == 2 else [(a, b)] if m == 1 else []):
            got[d] = got.get(d, 0) + 1
    return got


@pytest.mark.parametrize("seed", range(6))
def test_every_directed_pair_once_on_any_lists(seed):
    rng = np.random.default_rng(seed)
    n = 40
    # a symmetric relation with its diagonal, then some mirrors removed
    m = rng.random((n, n)) < 0.15
    m = m | m.T | np.eye(n, dtype=bool)
    drop = rng.random((n, n)) < 0.3
    m &= ~(drop & ~np.eye(n, dtype=bool))
    records = np.argwhere(m)   # target-major, sources ascending, as the library sorts them
    got = evaluated(records)
    want = {(int(a), int(b)) for a, b in records if a != b}
    assert set(got) == want
    assert all(v == 1 for v in got.values())
    # both kinds of record occur: mutual pairs and one-way ones
    md = modes(records)
    assert 2 in md and 1 in md


def test_rule_on_a_planted_mistake_fails():
    """The coverage check catches a plausible slip in the rule: the b < a
    records skipped whether or not the mirror exists."""
    records = np.array([[0, 0], [0, 1], [1, 1], [2, 0], [2, 2]])   # 2 <- 0 has no mirror

    def wrong(recs):
        return [0 if a == b or b < a else (2 if (b, a) in set(map(tuple, recs)) else 1) for a, b in recs]

    got = {}
    for (a, b), m in zip(map(tuple, records), wrong(records)):
        for d in ([(a, b), (b, a)] if m == 2 else [(a, b)] if m == 1 else []):
            got[d] = got.get(d, 0) + 1
    assert (2, 0) not in got                      # the wrong rule loses a pair
    assert (2, 0) in evaluated(records)           # the stated rule keeps it


@pytest.mark.parametrize("name,n,leaf,theta", [("uniform", 20000, 32, 0.5), ("plummer", 30000, 64, 0.4),
                                               ("clustered", 30000, 64, 0.5), ("clustered", 20000, 8, 0.6)])
def test_dual_traversal_lists_are_symmetric(name, n, leaf, theta):
    wl = W.make_workload(name, n=n)
    t = O.build_tree(wl.pos, leaf, theta)
    pairs = set(map(tuple, t.p2p.tolist()))
    assert all((b, a) in pairs for a, b in pairs)
    # so every cross-leaf record is evaluated by the mutual form, once, from its lower leaf
    md = modes(t.p2p)
    cross = t.p2p[:, 0] != t.p2p[:, 1]
    assert set(np.asarray(md)[cross].tolist()) == {0, 2}
    assert sum(1 for x in md if x == 2) * 2 == int(cross.sum())
