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
source type an FMM form of this gradient needs besides charges.
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
