"""Pins for the CPU oracle: facts fixed by the mathematics of the Laplace FMM.

The paper prints no worked example, no coefficients and no accuracy figures,
so nothing here is a value from the paper.  Every pin below is a closed form,
an invariant, an exact identity, a classical error bound, or brute force on a
tiny input.  Each pin is a plain function that raises AssertionError; the
pytest wrappers call them against the real oracle, and the planted-mistake
test calls them against oracle builds with a deliberate error to show that
some pin catches each error.
"""
from __future__ import annotations

import math

import numpy as np

import oracle as O
import workloads as W


def _rng(seed):
    return np.random.default_rng(seed)


# ---------------------------------------------------------------- direct sum

def pin_direct_two_charges():
    """Two charges: phi_0 = q_1 / r, grad phi_0 = -q_1 (x_0 - x_1) / r^3."""
    pos = np.array([[0.0, 0.0, 0.0], [3.0, 4.0, 0.0]])
    q = np.array([2.0, -0.5])
    phi, g = O.direct(pos, q)
    assert phi[0] == -0.5 / 5.0 and phi[1] == 2.0 / 5.0
    assert np.allclose(g[0], 0.5 * np.array([-3.0, -4.0, 0.0]) / 125.0, rtol=1e-15, atol=0)
    assert np.allclose(g[1], -2.0 * np.array([3.0, 4.0, 0.0]) / 125.0, rtol=1e-15, atol=0)


def pin_direct_cube_corners():
    """Unit charges on the corners of a cube of side a: by symmetry each corner
    sees 3 charges at a, 3 at a*sqrt2, 1 at a*sqrt3, and the gradient points
    along the body diagonal into the cube with |component| = (1 + 1/sqrt2 +
    1/(3 sqrt3)) / a^2."""
    a = 0.75
    pos = np.array([[i, j, k] for i in (0, 1) for j in (0, 1) for k in (0, 1)], float) * a
    phi, g = O.direct(pos, np.ones(8))
    expect = (3.0 + 3.0 / math.sqrt(2) + 1.0 / math.sqrt(3)) / a
    assert np.allclose(phi, expect, rtol=1e-15)
    gmag = (1.0 + 1.0 / math.sqrt(2) + 1.0 / (3.0 * math.sqrt(3))) / a ** 2
    inward = (0.5 * a - pos) / (0.5 * a)  # +-1 per component, pointing to the centre
    assert np.allclose(g, gmag * inward, rtol=1e-14)


def pin_direct_coincident_and_third_law():
    """r = 0 pairs are skipped; sum_i q_i grad phi_i = 0 (Newton's third law)."""
    rng = _rng(1)
    pos = rng.random((50, 3))
    pos[7] = pos[3]
    q = rng.uniform(-1, 1, 50)
    phi, g = O.direct(pos, q)
    assert np.all(np.isfinite(phi)) and np.all(np.isfinite(g))
    net = (q[:, None] * g).sum(0)
    assert np.abs(net).max() < 1e-12 * np.abs(q[:, None] * g).sum()
    # homogeneity: scaling positions by 2 halves phi exactly, quarters grad
    phi2, g2 = O.direct(2.0 * pos, q)
    assert np.array_equal(phi2, 0.5 * phi) and np.array_equal(g2, 0.25 * g)


# ---------------------------------------------------------------- operators

def _classical_bound(rs, rx, p, qabs=1.0):
    """|1/|x-y| - order-p multipole| <= qabs (rs/rx)^(p+1) / (rx - rs)."""
    return qabs * (rs / rx) ** (p + 1) / (rx - rs)


def pin_multipole_single_charge():
    """P2M of one charge then M2P far away: error within the classical bound,
    and far from zero error (so the expansion is truncated where it should be)."""
    rng = _rng(2)
    for p in range(0, 13):
        for _ in range(4):
            y = rng.normal(size=3); y *= 0.3 * rng.random() / np.linalg.norm(y)
            x = rng.normal(size=3); x *= (1.0 + rng.random()) / np.linalg.norm(x)
            M = O.p2m(p, np.zeros(3), y[None, :], np.array([1.0]))
            err = abs(O.m2p(p, M, x) - 1.0 / np.linalg.norm(x - y))
            assert err <= _classical_bound(np.linalg.norm(y), np.linalg.norm(x), p) * (1 + 1e-9) + 1e-15


def pin_multipole_on_axis():
    """On the z axis the multipole of a charge at (0,0,a) is the Legendre series
    1/(z - a) = sum a^n / z^(n+1): the order-p truncation is the geometric sum."""
    a, z = 0.25, 2.0
    for p in range(0, 10):
        M = O.p2m(p, np.zeros(3), np.array([[0.0, 0.0, a]]), np.array([1.0]))
        got = O.m2p(p, M, np.array([0.0, 0.0, z]))
        exact = sum(a ** n / z ** (n + 1) for n in range(p + 1))
        assert abs(got - exact) < 1e-15 * exact * (p + 2)


def pin_m2m_exact():
    """M2M is exact at every order: shifting the child expansion to the parent
    centre equals P2M at the parent centre."""
    rng = _rng(3)
    for p in (0, 1, 2, 5, 8, 10):
        pos = rng.random((20, 3)) * 0.5
        q = rng.uniform(-1, 1, 20)
        cc, cp = np.array([0.25, 0.25, 0.25]), np.array([0.5, 0.5, 0.5])
        Mc = O.p2m(p, cc, pos, q)
        Mp = O.p2m(p, cp, pos, q)
        Mt = O.m2m(p, Mc, cc - cp)
        assert np.abs(Mt - Mp).max() <= 1e-13 * max(1.0, np.abs(Mp).max())


def pin_l2l_exact():
    """L2L is exact: the shifted local expansion evaluates to the same potential
    and gradient at every point."""
    rng = _rng(4)
    for p in (1, 3, 6, 9):
        L = rng.normal(size=O.ncoef(p)) + 1j * rng.normal(size=O.ncoef(p))
        # make it the expansion of a real field: L_n^{-m} = (-1)^m conj(L_n^m)
        for n in range(p + 1):
            L[O.hidx(n, 0)] = L[O.hidx(n, 0)].real
            for m in range(1, n + 1):
                L[O.hidx(n, -m)] = (-1) ** m * np.conj(L[O.hidx(n, m)])
        d = rng.normal(size=3) * 0.2
        Lc = O.l2l(p, L, d)
        for _ in range(3):
            x = rng.normal(size=3) * 0.2
            f0, g0 = O.l2p(p, L, x)
            f1, g1 = O.l2p(p, Lc, x - d)
            assert abs(f0 - f1) <= 1e-12 * (1 + abs(f0))
            assert np.abs(g0 - g1).max() <= 1e-12 * (1 + np.abs(g0).max())


def pin_m2l_single_charge():
    """P2M -> M2L -> L2P of one charge reproduces 1/|x-y| and its gradient
    within a translation bound; with a reversed sign on odd local degrees, or a
    transposed operand, the field of a displaced charge is wrong at O(1)."""
    rng = _rng(5)
    for p in (2, 4, 8, 12):
        for _ in range(5):
            a = b = 0.5
            y = rng.uniform(-a, a, 3) / math.sqrt(3)
            t = rng.normal(size=3); t *= 3.0 / np.linalg.norm(t)
            x = t + rng.uniform(-b, b, 3) / math.sqrt(3)
            M = O.p2m(p, np.zeros(3), y[None, :], np.array([1.0]))
            L = O.m2l(p, M, t)
            f, g = O.l2p(p, L, x - t)
            r = x - y
            R = np.linalg.norm(r)
            rho = (a + b) / 3.0
            bound = 4.0 * rho ** (p + 1) / (3.0 - a - b)
            assert abs(f - 1.0 / R) <= bound
            assert np.abs(g + r / R ** 3).max() <= 4.0 * bound * (p + 1)


def pin_m2l_order_zero():
    """p = 0: M2L of a total charge Q gives the local constant Q / |D| exactly."""
    rng = _rng(6)
    pos = rng.random((10, 3))
    q = rng.uniform(-1, 1, 10)
    M = O.p2m(0, np.zeros(3), pos, q)
    D = np.array([3.0, -4.0, 12.0])
    L = O.m2l(0, M, D)
    assert abs(L[0].real - q.sum() / 13.0) <= 1e-15 * abs(q.sum())
    assert L[0].imag == 0.0


def pin_l2p_gradient_fd():
    """L2P gradient equals the central difference of the L2P potential."""
    rng = _rng(7)
    p = 7
    M = O.p2m(p, np.zeros(3), rng.random((5, 3)) - 0.5, rng.uniform(-1, 1, 5))
    L = O.m2l(p, M, np.array([4.0, 1.0, -2.0]))
    x = np.array([0.1, -0.2, 0.05])
    f, g = O.l2p(p, L, x)
    h = 1e-5
    for d in range(3):
        e = np.zeros(3); e[d] = h
        fd = (O.l2p(p, L, x + e)[0] - O.l2p(p, L, x - e)[0]) / (2 * h)
        assert abs(fd - g[d]) <= 1e-8 * (1 + abs(g[d]))


# ---------------------------------------------------------------- tree + lists

def _decode(keys, bits):
    """Integer coordinates from interleaved keys of 3*bits bits."""
    keys = np.asarray(keys, np.uint64)
    k = np.zeros((keys.size, 3), np.int64)
    for b in range(bits):
        for d in range(3):
            k[:, d] |= ((keys >> np.uint64(3 * b + d)) & np.uint64(1)).astype(np.int64) << b
    return k


def pin_tree_invariants(pos, leaf_size=16, theta=0.5):
    T = O.build_tree(pos, leaf_size, theta)
    n = pos.shape[0]
    assert sorted(T.perm.tolist()) == list(range(n))
    assert np.all(np.diff(T.keys.astype(np.float64)) >= 0) and np.all(T.keys[1:] >= T.keys[:-1])
    # stable: equal keys keep input order
    same = T.keys[1:] == T.keys[:-1]
    assert np.all(T.perm[1:][same] > T.perm[:-1][same])
    # every particle lies in the cube of its own 21-bit key (bit order check)
    k = _decode(T.keys, 21)
    u = T.side / 2 ** 21
    x = pos[T.perm]
    lo = T.origin + k * u
    assert np.all(x >= lo - 1e-12 * T.side) and np.all(x <= lo + u + 1e-12 * T.side)
    # cells: root covers all, children partition parents, leaf rule, level order
    assert T.first[0] == 0 and T.count[0] == n and T.level[0] == 0
    assert np.all(np.diff(T.level) >= 0)
    for c in range(T.ncell):
        lv = int(T.level[c])
        if c > 0:
            par = T.parent[c]
            assert T.level[par] == lv - 1
            assert (T.cell_key[c] >> np.uint64(3)) == T.cell_key[par]
        if T.child_count[c]:
            cf, cn = T.child_first[c], T.child_count[c]
            assert T.count[cf:cf + cn].sum() == T.count[c]
            assert T.first[cf] == T.first[c]
            assert T.count[c] > leaf_size and lv < 21
        else:
            assert T.count[c] <= leaf_size or lv == 21
        # every particle of the cell carries the cell's key prefix
        sh = np.uint64(3 * (21 - lv))
        ks = T.keys[T.first[c]:T.first[c] + T.count[c]] >> sh
        assert np.all(ks == T.cell_key[c])
    same_level = T.level[1:] == T.level[:-1]
    assert np.all(T.cell_key[1:][same_level] > T.cell_key[:-1][same_level])
    return T


def _cell_size_twoc(T):
    s = (np.int64(1) << (21 - T.level.astype(np.int64)))
    kc = np.zeros((T.ncell, 3), np.int64)
    for c in range(T.ncell):
        kc[c] = _decode(np.array([T.cell_key[c]]), int(T.level[c]))[0]
    return s, 2 * kc * s[:, None] + s[:, None]


def pin_lists_cover_every_pair_once(pos, leaf_size=16, theta=0.5):
    """Every ordered particle pair (i, j) -- including i == j -- is covered by
    exactly one emitted pair (A contains i, B contains j), P2P or M2L; every M2L
    pair passes the acceptance test; every P2P pair is leaf-leaf and fails it."""
    T = O.build_tree(pos, leaf_size, theta)
    n = pos.shape[0]
    inv = np.empty(n, np.int64)
    inv[T.perm] = np.arange(n)
    cover = np.zeros((n, n), np.int16)
    s, twoc = _cell_size_twoc(T)

    def accept(a, b):
        D = twoc[a] - twoc[b]
        return float((s[a] + s[b]) ** 2) < (theta * theta) * float((D * D).sum())

    for kind, lst in (("m2l", T.m2l), ("p2p", T.p2p)):
        for a, b in lst:
            if kind == "m2l":
                assert accept(a, b)
            else:
                assert T.child_count[a] == 0 and T.child_count[b] == 0 and not accept(a, b)
            ra = slice(T.first[a], T.first[a] + T.count[a])
            rb = slice(T.first[b], T.first[b] + T.count[b])
            cover[np.ix_(np.arange(n)[ra], np.arange(n)[rb])] += 1
    assert np.all(cover == 1), (np.argwhere(cover != 1)[:5])
    # lists are sorted and unique
    for lst in (T.m2l, T.p2p):
        if len(lst) > 1:
            key = lst[:, 0].astype(np.int64) * (1 << 32) + lst[:, 1]
            assert np.all(np.diff(key) > 0)
    return T


def pin_scaling_invariance():
    """Scaling positions by 2^s leaves keys and lists unchanged and scales phi by 2^-s."""
    wl = W.make_workload("plummer", n=3000)
    T1 = O.build_tree(wl.pos, 32, 0.5)
    T2 = O.build_tree(wl.pos * 8.0, 32, 0.5)
    assert np.array_equal(T1.keys, T2.keys) and np.array_equal(T1.m2l, T2.m2l)
    assert np.array_equal(T1.p2p, T2.p2p) and np.array_equal(T1.perm, T2.perm)
    f1, g1 = T1.evaluate(5, wl.q)
    f2, g2 = T2.evaluate(5, wl.q)
    assert np.abs(f2 * 8.0 - f1).max() <= 1e-14 * np.abs(f1).max()
    assert np.abs(g2 * 64.0 - g1).max() <= 1e-13 * np.abs(g1).max()


# ---------------------------------------------------------------- whole FMM

def pin_fmm_equals_direct_without_far_field():
    """Nothing accepted (theta tiny) or one leaf: the FMM is the direct sum."""
    wl = W.make_workload("uniform", n=700)
    pd, gd = O.direct(wl.pos, wl.q)
    T = O.build_tree(wl.pos, 16, 1e-6)
    assert len(T.m2l) == 0
    f, g = T.evaluate(4, wl.q)
    assert O.rel_l2(f, pd) <= 1e-13 and O.rel_l2(g, gd) <= 1e-13
    f, g = O.fmm_evaluate(wl.pos, wl.q, p=3, leaf_size=1000, theta=0.5)
    assert O.rel_l2(f, pd) <= 1e-13 and O.rel_l2(g, gd) <= 1e-13


def pin_fmm_error_decays_with_p():
    """The FMM error against the direct sum decays geometrically in p."""
    wl = W.make_workload("uniform", n=2000)
    pd, gd = O.direct(wl.pos, wl.q)
    T = O.build_tree(wl.pos, 16, 0.5)
    ps = list(range(0, 13, 2))
    errs = [O.rel_l2(T.evaluate(p, wl.q, nthreads=4)[0], pd) for p in ps]
    slope = np.polyfit(ps, np.log(errs), 1)[0]
    assert slope < -0.3, (errs, slope)
    assert all(errs[i + 1] < errs[i] for i in range(len(errs) - 1)), errs
    assert errs[-1] < 1e-5


def pin_fmm_high_order_matches_direct():
    """Tiny input, high order: FMM and brute force agree to near rounding."""
    wl = W.make_workload("clustered", n=400)
    pd, gd = O.direct(wl.pos, wl.q)
    f, g = O.fmm_evaluate(wl.pos, wl.q, p=20, leaf_size=8, theta=0.3)
    assert O.rel_l2(f, pd) <= 1e-9 and O.rel_l2(g, gd) <= 1e-8


def pin_fmm_net_force():
    """The net force sum_i q_i grad phi_i vanishes to the FMM error level."""
    wl = W.make_workload("plummer", n=3000)
    pd, gd = O.direct(wl.pos, wl.q)
    f, g = O.fmm_evaluate(wl.pos, wl.q, p=8, leaf_size=32, theta=0.4)
    tot = np.abs(wl.q[:, None] * gd).sum()
    assert np.abs((wl.q[:, None] * g).sum(0)).max() <= 1e-4 * tot


def pin_fmm_sampled_matches_full():
    """The per-leaf sampled evaluation equals the full evaluation."""
    wl = W.make_workload("clustered", n=3000)
    T = O.build_tree(wl.pos, 32, 0.5)
    f, g = T.evaluate(6, wl.q)
    leaves = np.nonzero(T.is_leaf)[0][::3]
    idx, fs, gs = T.evaluate_leaves(6, wl.q, leaves)
    assert np.abs(fs - f[idx]).max() <= 1e-13 * np.abs(f).max()
    assert np.abs(gs - g[idx]).max() <= 1e-13 * np.abs(g).max()


def _tiny_sets():
    out = []
    for name in ("uniform", "plummer", "clustered"):
        out.append((name, W.make_workload(name, n=1500).pos))
    return out


ALL_PINS = [
    pin_direct_two_charges, pin_direct_cube_corners, pin_direct_coincident_and_third_law,
    pin_multipole_single_charge, pin_multipole_on_axis, pin_m2m_exact, pin_l2l_exact,
    pin_m2l_single_charge, pin_m2l_order_zero, pin_l2p_gradient_fd,
    lambda: [pin_tree_invariants(p) for _, p in _tiny_sets()],
    lambda: [pin_lists_cover_every_pair_once(p) for _, p in _tiny_sets()[:2]],
    pin_scaling_invariance, pin_fmm_equals_direct_without_far_field, pin_fmm_error_decays_with_p,
    pin_fmm_high_order_matches_direct, pin_fmm_net_force, pin_fmm_sampled_matches_full,
]


# ---------------------------------------------------------------- gradients (O9)

def pin_direct_gradient_formulas():
    """For L = sum_i w_i phi_i: dL/dq_j = phi^(w)_j and
    dL/dx_k = w_k grad phi^(q)(x_k) + q_k grad phi^(w)(x_k), against central
    differences of L computed by the direct sum."""
    rng = _rng(8)
    n = 40
    pos = rng.random((n, 3))
    q = rng.normal(size=n)
    w = rng.normal(size=n)

    def loss(x, qq):
        return float(np.dot(w, O.direct(x, qq)[0]))

    phi_w, g_w = O.direct(pos, w)
    _, g_q = O.direct(pos, q)
    dq = phi_w
    dx = w[:, None] * g_q + q[:, None] * g_w
    h = 1e-6
    for j in (0, 7, 39):
        e = np.zeros(n); e[j] = h
        fd = (loss(pos, q + e) - loss(pos, q - e)) / (2 * h)
        assert abs(fd - dq[j]) <= 1e-7 * (1 + abs(dq[j]))
        for d in range(3):
            xp, xm = pos.copy(), pos.copy()
            xp[j, d] += h; xm[j, d] -= h
            fd = (loss(xp, q) - loss(xm, q)) / (2 * h)
            assert abs(fd - dx[j, d]) <= 1e-6 * (1 + abs(dx[j, d]))


def pin_fmm_gradient_fixed_tree():
    """With the tree held fixed (cells and centres from the unperturbed
    positions), the FMM loss is smooth in x; at high order its central
    difference matches w grad phi^(q) + q grad phi^(w) from two FMM passes."""
    wl = W.make_workload("gradient", n=1500)
    pos, q, w = wl.pos, wl.q, wl.extra["w"]
    T = O.build_tree(pos, 32, 0.5)
    p = 16
    phi_q, g_q = T.evaluate(p, q, nthreads=4)
    phi_w, g_w = T.evaluate(p, w, nthreads=4)
    dx = w[:, None] * g_q + q[:, None] * g_w

    def loss(x):
        T.pos = np.ascontiguousarray(x)
        return float(np.dot(w, T.evaluate(p, q, nthreads=4)[0]))

    h = 1e-6
    for j in (3, 500, 1499):
        for d in range(3):
            xp, xm = pos.copy(), pos.copy()
            xp[j, d] += h; xm[j, d] -= h
            fd = (loss(xp) - loss(xm)) / (2 * h)
            assert abs(fd - dx[j, d]) <= 1e-5 * np.abs(dx).max()
    T.pos = pos


# ---------------------------------------------------------------- hand-worked tree cases

def pin_root_cube_centred():
    """Root cube of two particles with unequal extents, worked by hand.

    Points (0, 0, 0) and (4, 2, 1): extents 4, 2, 1, so side = 4 (the longest)
    and the cube is centred on the bounding box in every axis: origin =
    (lo + hi)/2 - side/2 = (0, -1, -1.5).  With u = side / 2^21 = 2^-19:
      (0, 0, 0): k = (0, 1 / 2^-19, 1.5 / 2^-19) = (0, 2^19, 2^19 + 2^18);
      (4, 2, 1): k = (2^21 clamped to 2^21 - 1, 3 * 2^19, 2.5 * 2^19)
                   = (2^21 - 1, 2^20 + 2^19, 2^20 + 2^18).
    Morton key bits: x bit b at 3b, y bit b at 3b + 1, z bit b at 3b + 2, so
      key(0,0,0) = 2^(3*19+1) + 2^(3*19+2) + 2^(3*18+2) = 2^58 + 2^59 + 2^56,
      key(4,2,1) = sum_b 2^(3b) (b = 0..20) + 2^61 + 2^58 + 2^62 + 2^56.
    A cube anchored at the low corner (origin = lo) or sides per axis would
    give other origins and keys."""
    T = O.build_tree(np.array([[0.0, 0.0, 0.0], [4.0, 2.0, 1.0]]), 1, 0.5)
    assert T.side == 4.0
    assert np.array_equal(T.origin, np.array([0.0, -1.0, -1.5]))
    k0 = (1 << 58) + (1 << 59) + (1 << 56)
    k1 = sum(1 << (3 * b) for b in range(21)) + (1 << 61) + (1 << 58) + (1 << 62) + (1 << 56)
    assert sorted(int(k) for k in T.keys) == sorted([k0, k1])
    # octants at level 1 (key bits 62, 61, 60): 0 for the first point, 7 for the second
    assert T.ncell == 3 and np.array_equal(T.level, [0, 1, 1])
    assert np.array_equal(T.cell_key, np.array([0, 0, 7], np.uint64))


def pin_traversal_tie_break():
    """Lists of four particles, worked by hand (leaf size 1, theta = 0.5).

    p0 = (0,0,0), p1 = (3/8)(1,1,1), p2 = (5/8)(1,1,1), p3 = (1,1,1): the root
    cube is [0,1]^3; cells in (level, key) order are the root 0, its octants
    c0 = [0,1/2]^3 (cell 1) and c7 = [1/2,1]^3 (cell 2), and the level-2
    leaves x000 = [0,1/4]^3 (3, holds p0), x111 = [1/4,1/2]^3 (4, p1),
    y000 = [1/2,3/4]^3 (5, p2), y111 = [3/4,1]^3 (6, p3).  Accept iff
    (s_i + s_j)^2 < theta^2 |2 (c_i - c_j)|^2 (sides s, in root units).
    (root, root) and (c0, c7) are rejected; cells of equal size split the
    target, so (c0, c7) becomes (x000, c7) -- accepted: 0.75^2 < 0.25 * 3 *
    1.25^2 -- and (x111, c7), rejected (0.25 * 3 * 0.75^2 < 0.75^2) with a leaf
    target, so the source splits: (x111, y111) is accepted (0.5^2 < 0.25 * 3)
    and (x111, y000) is P2P.  Symmetrically (y111, c0) is accepted and
    (y000, x000) too.  Splitting the source on equal size would give (c0, y111)
    and (c7, x000) instead."""
    pos = np.array([[0.0] * 3, [0.375] * 3, [0.625] * 3, [1.0] * 3])
    T = O.build_tree(pos, 1, 0.5)
    assert T.ncell == 7
    assert np.array_equal(T.level, [0, 1, 1, 2, 2, 2, 2])
    assert np.array_equal(T.count, [4, 2, 2, 1, 1, 1, 1])
    assert np.array_equal(T.m2l, np.array([[3, 2], [4, 6], [5, 3], [6, 1]], np.int32))
    assert np.array_equal(T.p2p, np.array([[3, 3], [3, 4], [4, 3], [4, 4], [4, 5], [5, 4], [5, 5], [5, 6],
                                           [6, 5], [6, 6]], np.int32))


def pin_split_rule_invariants(pos, leaf_size=8, theta=0.5):
    """Consequences of the split rule (split the larger cell; the target on
    equal size or when the source is a leaf): a pair whose source is finer than
    its target has a leaf target, and a pair whose target is more than one
    level finer than its source has a leaf source."""
    T = O.build_tree(pos, leaf_size, theta)
    leaf = T.is_leaf
    for lst in (T.m2l, T.p2p):
        if len(lst) == 0:
            continue
        lt, ls = T.level[lst[:, 0]], T.level[lst[:, 1]]
        assert np.all(leaf[lst[ls > lt, 0]])
        assert np.all(leaf[lst[lt > ls + 1, 1]])
