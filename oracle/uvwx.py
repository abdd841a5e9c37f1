"""Parent-neighbour-child interaction lists (U, V, W, X) and the FMM evaluated
through them (potential and its gradient) -- TEST INFRASTRUCTURE (oracle).

Section 2.1 of the paper names two ways to decide which cells are well
separated: the size/distance ratio (the dual traversal of the rest of the
oracle) and the parent-neighbour-child relationship of the adaptive octree,
for which it refers to Cheng, Greengard and Rokhlin (1999).  This module
restates the lists of that second approach from their definitions, by brute
force over the boxes of a small tree, and evaluates the FMM through them:

* two boxes are *adjacent* when neither contains the other and their closed
  cubes share at least one point; the *neighbours* of a box are the adjacent
  boxes of its own level;
* U(B), B a leaf: B and every leaf adjacent to B (direct sum);
* V(B): the children of B's parent's neighbours that are not adjacent to B
  (multipole to local);
* W(B), B a leaf: the boxes D finer than B, not adjacent to B, whose parent is
  adjacent to B (the multipole of D evaluated at B's particles);
* X(B): the leaves A with B in W(A) (A's particles into B's local expansion).

Evaluation: P2M at the leaves and M2M upwards; the local expansion of every
box gathers M2L from V(B) and the particles of X(B) (a particle's multipole
about its own position is its charge alone, so its local expansion is the
M2L of that monopole, exact up to the order p); L2L downwards; at a leaf the
local expansion, the direct sum over U(B) and the multipoles of W(B) give the
potential and its gradient.  A multipole is evaluated at a point x as the M2L
to a local expansion about x read at x itself: its order-0 and order-1 terms
sum every multipole term exactly, so this is the multipole's field and field
gradient at x.  Every directed pair of particles is accounted for exactly once
(``coverage`` checks it), and the result tends to the direct sum as p grows.
Pure-Python loops over boxes: small trees only (a few thousand particles).
"""
from __future__ import annotations

import numpy as np

from . import build_tree, l2l, l2p, m2l, m2m, ncoef, p2m


class Boxes:
    """Integer geometry of an oracle tree's cells: box b spans
    [lo_b, lo_b + s_b] on every axis in units of side / 2^21."""

    def __init__(self, tree):
        self.t = tree
        nc = tree.ncell
        kc = np.zeros((nc, 3), dtype=np.int64)
        for b in range(21):
            for d in range(3):
                kc[:, d] |= ((tree.cell_key >> np.uint64(3 * b + d)) & np.uint64(1)).astype(np.int64) << b
        self.size = np.int64(1) << (21 - tree.level.astype(np.int64))
        self.lo = kc * self.size[:, None]
        self.hi = self.lo + self.size[:, None]
        self.centre = tree.centres()
        self.leaf = tree.child_count == 0
        self.children = [list(range(tree.child_first[c], tree.child_first[c] + tree.child_count[c]))
                         if tree.child_count[c] > 0 else [] for c in range(nc)]
        self.by_level = {}
        for c in range(nc):
            self.by_level.setdefault(int(tree.level[c]), []).append(c)

    def contains(self, a, b):
        """Box a contains box b (or is b)."""
        return bool(np.all(self.lo[a] <= self.lo[b]) and np.all(self.hi[b] <= self.hi[a]))

    def adjacent(self, a, b):
        if a == b or self.contains(a, b) or self.contains(b, a):
            return False
        return bool(np.all(self.lo[a] <= self.hi[b]) and np.all(self.lo[b] <= self.hi[a]))

    def neighbours(self, b):
        return [c for c in self.by_level[int(self.t.level[b])] if self.adjacent(b, c)]

    def descendants(self, b):
        out, stack = [], list(self.children[b])
        while stack:
            c = stack.pop()
            out.append(c)
            stack.extend(self.children[c])
        return out


def build_lists(tree):
    """U, V, W, X of every box (dicts box -> sorted list), from the definitions."""
    bx = Boxes(tree)
    nc = tree.ncell
    U, V, W, X = {}, {}, {}, {c: [] for c in range(nc)}
    leaves = [c for c in range(nc) if bx.leaf[c]]
    for b in range(nc):
        par = int(tree.parent[b])
        if par >= 0:
            V[b] = sorted(c for nb in bx.neighbours(par) for c in bx.children[nb] if not bx.adjacent(b, c))
        else:
            V[b] = []
    for b in leaves:
        U[b] = sorted([b] + [a for a in leaves if bx.adjacent(a, b)])
        w = []
        for nb in bx.neighbours(b):
            for d in bx.descendants(nb):
                if not bx.adjacent(b, d) and bx.adjacent(int(tree.parent[d]), b):
                    w.append(d)
        W[b] = sorted(w)
        for d in w:
            X[d].append(b)
    for c in range(nc):
        X[c] = sorted(X[c])
    return bx, U, V, W, X


def coverage(tree, lists=None):
    """cov[t, i] = how many times the particles of target leaf t reach source
    particle i through the lists (U directly, V and X through t's ancestors'
    local expansions, W through multipoles).  Exactly 1 everywhere for a
    correct set of lists."""
    bx, U, V, W, X = lists if lists is not None else build_lists(tree)
    n = tree.n
    first, count = tree.first, tree.count
    leaves = [c for c in range(tree.ncell) if bx.leaf[c]]
    cov = np.zeros((len(leaves), n), dtype=np.int64)

    def add(row, c):
        cov[row, first[c]:first[c] + count[c]] += 1

    for row, t in enumerate(leaves):
        for a in U[t]:
            add(row, a)
        for d in W[t]:
            add(row, d)
        anc = t
        while anc >= 0:
            for c in V[anc]:
                add(row, c)
            for a in X[anc]:
                add(row, a)
            anc = int(tree.parent[anc])
    return leaves, cov


def pair_lists(tree, lists=None):
    """The lists as (target, source) pairs with W and X taken as direct sums:
    M2L pairs = V; P2P pairs = U, plus (b, L) and (L, b) for every leaf L
    inside a box D of W(b) (X is the dual of W).  Both sorted by (target,
    source); every P2P pair joins two leaves and the P2P relation is
    symmetric."""
    bx, U, V, W, X = lists if lists is not None else build_lists(tree)
    m2l_pairs = sorted((b, c) for b in V for c in V[b])
    p2p = set((b, a) for b in U for a in U[b])
    for b, ws in W.items():
        for d in ws:
            for leaf in ([d] if bx.leaf[d] else [c for c in bx.descendants(d) if bx.leaf[c]]):
                p2p.add((b, leaf))
                p2p.add((leaf, b))
    return (np.array(m2l_pairs, dtype=np.int32).reshape(-1, 2),
            np.array(sorted(p2p), dtype=np.int32).reshape(-1, 2))


def evaluate(pos, q, p: int, leaf_size: int = 16, theta: float = 0.5, tree=None, lists=None, wx: str = "expansions"):
    """(phi [n], grad phi [n, 3]) of every particle, input order, through the
    U/V/W/X lists.  wx = "expansions": W by multipoles at the particles, X by
    local expansions (Cheng et al.); wx = "direct": both by direct sums between
    the leaves involved (``pair_lists``).  theta only shapes the oracle tree's
    construction call; the lists use adjacency alone."""
    if wx not in ("expansions", "direct"):
        raise ValueError("wx must be 'expansions' or 'direct'")
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.float64)
    tree = tree if tree is not None else build_tree(pos, leaf_size, theta)
    bx, U, V, W, X = lists if lists is not None else build_lists(tree)
    if wx == "direct":
        _, pp = pair_lists(tree, (bx, U, V, W, X))
        U = {}
        for b, a in pp:
            U.setdefault(int(b), []).append(int(a))
        W = {b: [] for b in W}
        X = {c: [] for c in X}
    nc, K = tree.ncell, ncoef(p)
    sp = pos[tree.perm]          # sorted positions
    sq = q[tree.perm]
    first, count = tree.first, tree.count
    ctr = bx.centre
    # upward: P2M at the leaves, M2M from the finest level up
    M = np.zeros((nc, K), dtype=np.complex128)
    order = np.argsort(-tree.level, kind="stable")
    for c in order:
        if bx.leaf[c]:
            sl = slice(first[c], first[c] + count[c])
            M[c] = p2m(p, ctr[c], sp[sl], sq[sl])
        else:
            for ch in bx.children[c]:
                M[c] += m2m(p, M[ch], ctr[ch] - ctr[c])
    # local expansions: V by M2L, X by the particles' monopoles, then L2L down
    L = np.zeros((nc, K), dtype=np.complex128)
    mono = np.zeros(K, dtype=np.complex128)
    for b in range(nc):
        for c in V[b]:
            L[b] += m2l(p, M[c], ctr[b] - ctr[c])
        for a in X[b]:
            for j in range(first[a], first[a] + count[a]):
                mono[0] = sq[j]
                L[b] += m2l(p, mono, ctr[b] - sp[j])
    for c in np.argsort(tree.level, kind="stable"):
        par = int(tree.parent[c])
        if par >= 0:
            L[c] += l2l(p, L[par], ctr[c] - ctr[par])
    # at the leaves: local expansion + U direct + W multipoles
    phi_sorted = np.zeros(tree.n)
    grad_sorted = np.zeros((tree.n, 3))
    zero = np.zeros(3)
    for t in range(nc):
        if not bx.leaf[t]:
            continue
        for i in range(first[t], first[t] + count[t]):
            v, g = l2p(p, L[t], sp[i] - ctr[t])
            for a in U[t]:
                for j in range(first[a], first[a] + count[a]):
                    dv = sp[i] - sp[j]
                    r = np.sqrt(np.sum(dv * dv))
                    if r > 0:
                        v += sq[j] / r
                        g = g - sq[j] * dv / r ** 3
            for d in W[t]:
                vw, gw = l2p(p, m2l(p, M[d], sp[i] - ctr[d]), zero)
                v += vw
                g = g + gw
            phi_sorted[i] = v
            grad_sorted[i] = g
    phi = np.zeros(tree.n)
    grad = np.zeros((tree.n, 3))
    phi[tree.perm] = phi_sorted
    grad[tree.perm] = grad_sorted
    return phi, grad
