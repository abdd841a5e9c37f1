"""Gradient of a loss on potentials and forces, by the direct sum -- TEST
INFRASTRUCTURE (oracle).

The FMM of Section 2.1 approximates phi_i = sum_{j != i} q_j / r_ij and the
force F_i = -q_i grad phi_i = q_i sum_j q_j (x_i - x_j) / r_ij^3.  For a loss

    L = sum_i a_i phi_i + sum_i b_i . F_i      (a: n, b: n x 3)

this module gives dL/dq and dL/dx in closed form, pair by pair (pairs at
distance 0 skipped, like the direct sum).  With d = x_i - x_j, r = |d|:

    d(1/r)/dx_i = -d / r^3                      (and + for x_j)
    d(d / r^3)/dx_i = T(d) = I / r^3 - 3 d d^T / r^5   (and -T for x_j)

so, summing over ordered pairs (i, j), i != j:

    dL/dq_k = sum_{i != k} a_i / r_ik  +  b_k . sum_j q_j d_kj / r_kj^3  +  sum_{i != k} q_i b_i . d_ik / r_ik^3
    dL/dx_k = -a_k sum_j q_j d_kj / r^3  +  q_k sum_i a_i d_ik / r^3
              + q_k sum_j q_j T(d_kj) b_k  -  q_k sum_i q_i T(d_ik) b_i

(the second and fourth terms are the reactions on k as a source).  Rows of
pairs are processed in blocks, so a few thousand particles stay in memory.
``dipole_direct`` gives the potential and gradient of point dipoles, the
source type an FMM form of this gradient needs besides charges;
``p2m_dipole`` their multipole, ``dipole_fmm`` their FMM through the oracle
tree's lists, and ``fmm_gradient`` the whole gradient through the FMM (one
charge pass with the charges a, the forward pass, four dipole passes).
"""
from __future__ import annotations

import numpy as np


def loss(pos, q, a, b, phi, grad_phi):
    """L from given potentials and potential gradients (e.g. ``oracle.direct``)."""
    force = -np.asarray(q)[:, None] * np.asarray(grad_phi)
    return float(np.dot(a, phi) + np.sum(b * force))


def gradient(pos, q, a, b, block: int = 256):
    """(dL/dx [n, 3], dL/dq [n]) of the loss above, FP64."""
    pos = np.asarray(pos, np.float64).reshape(-1, 3)
    q = np.asarray(q, np.float64).ravel()
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).reshape(-1, 3)
    n = pos.shape[0]
    dx = np.zeros((n, 3))
    dq = np.zeros(n)
    for k0 in range(0, n, block):
        k1 = min(n, k0 + block)
        d = pos[k0:k1, None, :] - pos[None, :, :]          # d[k, j] = x_k - x_j
        r2 = np.sum(d * d, axis=-1)
        ok = r2 > 0
        rinv = np.where(ok, 1.0 / np.sqrt(np.where(ok, r2, 1.0)), 0.0)
        r3 = rinv ** 3
        r5 = rinv ** 5
        e = d * r3[..., None]                               # e[k, j] = d_kj / r^3
        eq = np.einsum("kjc,j->kc", e, q)                   # sum_j q_j d_kj / r^3 = -grad phi_k
        # dL/dq_k: potential of the charges a at k; b_k . (the sum above); the
        # term of every force F_i on k's charge, with d_ik = -d_ki
        dq[k0:k1] += rinv @ a
        dq[k0:k1] += np.einsum("kc,kc->k", b[k0:k1], eq)
        dq[k0:k1] -= np.einsum("kjc,jc,j->k", e, b, q)
        # dL/dx_k: a_k grad phi_k; k as the source of phi_i (d/dx_k of 1/r_ik = d_ik / r^3)
        dx[k0:k1] -= a[k0:k1, None] * eq
        dx[k0:k1] -= q[k0:k1, None] * np.einsum("kjc,j->kc", e, a)
        # F_k through x_k: q_k sum_j q_j T(d_kj) b_k; F_i through its source x_k:
        # -q_k sum_i q_i T(d_ik) b_i, and T is even in d
        db_k = np.einsum("kjc,kc->kj", d, b[k0:k1])
        tb_k = b[k0:k1, None, :] * r3[..., None] - 3.0 * d * (db_k * r5)[..., None]
        dx[k0:k1] += q[k0:k1, None] * np.einsum("kjc,j->kc", tb_k, q)
        db_i = np.einsum("kjc,jc->kj", d, b)
        tb_i = b[None, :, :] * r3[..., None] - 3.0 * d * (db_i * r5)[..., None]
        dx[k0:k1] -= q[k0:k1, None] * np.einsum("kjc,j->kc", tb_i, q)
    return dx, dq


def dipole_direct(pos, dip, block: int = 256):
    """Potential and its gradient at every particle of point dipoles dip_j at
    x_j (pairs at distance 0 skipped): psi_k = sum_j dip_j . d_kj / r^3,
    grad psi_k = sum_j T(d_kj) dip_j, d_kj = x_k - x_j.  A dipole p at x_j is
    the limit of the charge pair +-|p|/e at x_j +- (e/2) p/|p|, and its
    potential is p . grad_{x_j} (1 / |x - x_j|)."""
    pos = np.asarray(pos, np.float64).reshape(-1, 3)
    dip = np.asarray(dip, np.float64).reshape(-1, 3)
    n = pos.shape[0]
    psi = np.zeros(n)
    grad = np.zeros((n, 3))
    for k0 in range(0, n, block):
        k1 = min(n, k0 + block)
        d = pos[k0:k1, None, :] - pos[None, :, :]
        r2 = np.sum(d * d, axis=-1)
        ok = r2 > 0
        rinv = np.where(ok, 1.0 / np.sqrt(np.where(ok, r2, 1.0)), 0.0)
        r3, r5 = rinv ** 3, rinv ** 5
        pd = np.einsum("kjc,jc->kj", d, dip)
        psi[k0:k1] = np.sum(pd * r3, axis=1)
        grad[k0:k1] = np.einsum("kj,jc->kc", r3, dip) - 3.0 * np.einsum("kj,kjc->kc", pd * r5, d)
    return psi, grad


def p2m_dipole(p, centre, pos, dip):
    """Multipole expansion (the oracle's complex coefficients, index n*n + n + m)
    of point dipoles dip_j at pos_j about centre: M_n^m = sum_j dip_j . grad
    R_n^m(x_j - c).  The gradient of a regular solid harmonic is made of
    harmonics one order lower: dz R_n^m = R_{n-1}^m, (dx + i dy) R_n^m =
    -R_{n-1}^{m+1}, (dx - i dy) R_n^m = R_{n-1}^{m-1}, so
    dip . grad R_n^m = dz_ R_{n-1}^m - (dx_ - i dy_)/2 R_{n-1}^{m+1}
                       + (dx_ + i dy_)/2 R_{n-1}^{m-1}
    (a harmonic whose |m| exceeds its degree is zero).  The harmonics of each
    dipole's position are the unit-charge P2M of the order below."""
    from . import hidx, ncoef, p2m
    pos = np.asarray(pos, np.float64).reshape(-1, 3)
    dip = np.asarray(dip, np.float64).reshape(-1, 3)
    M = np.zeros(ncoef(p), dtype=np.complex128)
    if p == 0:
        return M
    for x, d in zip(pos, dip):
        Rl = p2m(p - 1, centre, x[None, :], np.ones(1))      # R_n^m(x - c), n <= p - 1

        def r(n, m):
            return Rl[hidx(n, m)] if abs(m) <= n else 0.0

        up, down = -(d[0] - 1j * d[1]) / 2.0, (d[0] + 1j * d[1]) / 2.0
        for n in range(1, p + 1):
            for m in range(-n, n + 1):
                M[hidx(n, m)] += d[2] * r(n - 1, m) + up * r(n - 1, m + 1) + down * r(n - 1, m - 1)
    return M


def dipole_fmm(tree, pos, dip, p: int):
    """Potential and gradient (input order) of point dipoles through the oracle
    tree's dual-traversal lists: dipole P2M at the leaves, M2M, M2L over the
    M2L pairs, L2L, then L2P plus the dipoles' direct terms over the P2P pairs
    -- the charge FMM of Section 2.1 with the dipole as the source type."""
    from . import l2l, l2p, m2l, m2m, ncoef
    pos = np.asarray(pos, np.float64).reshape(-1, 3)
    dip = np.asarray(dip, np.float64).reshape(-1, 3)
    nc, K = tree.ncell, ncoef(p)
    sp, sd = pos[tree.perm], dip[tree.perm]
    first, count = tree.first, tree.count
    ctr = tree.centres()
    leaf = tree.child_count == 0
    M = np.zeros((nc, K), dtype=np.complex128)
    for c in np.argsort(-tree.level, kind="stable"):
        if leaf[c]:
            sl = slice(first[c], first[c] + count[c])
            M[c] = p2m_dipole(p, ctr[c], sp[sl], sd[sl])
        else:
            for ch in range(tree.child_first[c], tree.child_first[c] + tree.child_count[c]):
                M[c] += m2m(p, M[ch], ctr[ch] - ctr[c])
    L = np.zeros((nc, K), dtype=np.complex128)
    for t, s_ in tree.m2l:
        L[t] += m2l(p, M[s_], ctr[t] - ctr[s_])
    for c in np.argsort(tree.level, kind="stable"):
        par = int(tree.parent[c])
        if par >= 0:
            L[c] += l2l(p, L[par], ctr[c] - ctr[par])
    psi = np.zeros(tree.n)
    grad = np.zeros((tree.n, 3))
    near = {}
    for t, s_ in tree.p2p:
        near.setdefault(int(t), []).append(int(s_))
    for t in np.nonzero(leaf)[0]:
        ti = np.arange(first[t], first[t] + count[t])
        for i in ti:
            psi[i], grad[i] = l2p(p, L[t], sp[i] - ctr[t])
        src = np.concatenate([np.arange(first[s_], first[s_] + count[s_]) for s_ in near.get(int(t), [])]) \
            if near.get(int(t)) else np.zeros(0, np.int64)
        if len(src):
            d = sp[ti, None, :] - sp[None, src, :]
            r2 = np.sum(d * d, axis=-1)
            ok = r2 > 0
            rinv = np.where(ok, 1.0 / np.sqrt(np.where(ok, r2, 1.0)), 0.0)
            r3, r5 = rinv ** 3, rinv ** 5
            pd = np.einsum("kjc,jc->kj", d, sd[src])
            psi[ti] += np.sum(pd * r3, axis=1)
            grad[ti] += np.einsum("kj,jc->kc", r3, sd[src]) - 3.0 * np.einsum("kj,kjc->kc", pd * r5, d)
    out_psi = np.zeros(tree.n)
    out_grad = np.zeros((tree.n, 3))
    out_psi[tree.perm] = psi
    out_grad[tree.perm] = grad
    return out_psi, out_grad


def fmm_gradient(tree, pos, q, a, b, p: int):
    """(dL/dx, dL/dq) of the loss above with every sum through the FMM of the
    oracle tree: one charge pass with the charges a, the forward pass, and
    four dipole passes (the dipoles -q_i b_i, and -q_j e_c for the columns of
    the Hessian), combined as dL/dq = phi^(a) + b . E + psi and
    dL/dx = a grad phi + q grad phi^(a) - q H b + q grad psi."""
    q = np.asarray(q, np.float64)
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64).reshape(-1, 3)
    phi, g = tree.evaluate(p, q)
    pha, ga = tree.evaluate(p, a)
    psi, gpsi = dipole_fmm(tree, pos, -q[:, None] * b, p)
    H = np.stack([dipole_fmm(tree, pos, -q[:, None] * np.eye(3)[c][None, :], p)[1] for c in range(3)], axis=2)
    hb = np.einsum("kic,kc->ki", H, b)
    dq = pha - np.einsum("kc,kc->k", b, g) + psi
    dx = a[:, None] * g + q[:, None] * ga - q[:, None] * hb + q[:, None] * gpsi
    return dx, dq
