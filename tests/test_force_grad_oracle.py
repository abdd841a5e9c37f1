"""Pins of the oracle's gradient of a loss on potentials and forces (the
backward a force-dependent loss needs), against quantities computed by the
oracle's C direct sum, which shares no code with it:

* central finite differences of L(x, q) in every coordinate and charge of a
  small system (L evaluated from ``oracle.direct``);
* with b = 0 the loss is linear in the potential, and its gradient is two
  direct sums: dL/dq = the potential of the charges a, dL/dx_k = a_k grad phi_k
  + q_k grad phi^(a)_k;
* the loss only depends on differences of positions, so dL/dx sums to zero.
A planted slip (a dropped source-side term) fails the finite differences."""
import numpy as np
import pytest

import oracle as O
from oracle import force_grad as FG


def _system(n, seed):
    rng = np.random.default_rng(seed)
    pos = rng.random((n, 3))
    q = rng.uniform(-1, 1, n)
    a = rng.standard_normal(n)
    b = rng.standard_normal((n, 3))
    return pos, q, a, b


def _loss(pos, q, a, b):
    phi, g = O.direct(pos, q)
    return FG.loss(pos, q, a, b, phi, g)


def _fd(pos, q, a, b, h=1e-6):
    n = len(q)
    dx = np.zeros((n, 3))
    dq = np.zeros(n)
    for k in range(n):
        for c in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[k, c] += h
            pm[k, c] -= h
            dx[k, c] = (_loss(pp, q, a, b) - _loss(pm, q, a, b)) / (2 * h)
        qp, qm = q.copy(), q.copy()
        qp[k] += h
        qm[k] -= h
        dq[k] = (_loss(pos, qp, a, b) - _loss(pos, qm, a, b)) / (2 * h)
    return dx, dq


@pytest.mark.parametrize("n,seed", [(12, 0), (40, 1)])
def test_matches_finite_differences(n, seed):
    pos, q, a, b = _system(n, seed)
    dx, dq = FG.gradient(pos, q, a, b, block=7)
    fx, fq = _fd(pos, q, a, b)
    assert np.max(np.abs(dx - fx)) <= 1e-6 * max(1.0, np.max(np.abs(fx)))
    assert np.max(np.abs(dq - fq)) <= 1e-6 * max(1.0, np.max(np.abs(fq)))


def test_potential_only_loss_is_two_direct_sums():
    pos, q, a, _ = _system(300, 2)
    dx, dq = FG.gradient(pos, q, a, np.zeros((300, 3)))
    phi_a, g_a = O.direct(pos, a)
    _, g_q = O.direct(pos, q)
    assert np.allclose(dq, phi_a, rtol=1e-12, atol=1e-12)
    assert np.allclose(dx, a[:, None] * g_q + q[:, None] * g_a, rtol=1e-10, atol=1e-10)


def test_translation_invariance_and_coincident_pairs():
    pos, q, a, b = _system(200, 3)
    pos[5] = pos[4]                     # a coincident pair contributes nothing, as in the direct sum
    dx, _ = FG.gradient(pos, q, a, b)
    assert np.all(np.isfinite(dx))
    assert np.linalg.norm(dx.sum(axis=0)) <= 1e-9 * np.abs(dx).sum()


def test_planted_slip_fails_finite_differences():
    pos, q, a, b = _system(12, 4)
    fx, _ = _fd(pos, q, a, b)
    src = open(FG.__file__).read()
    slip = src.replace("        dx[k0:k1] -= q[k0:k1, None] * np.einsum(\"kjc,j->kc\", tb_i, q)\n", "")
    assert slip != src
    ns = {}
    exec(compile(slip, "force_grad_slip", "exec"), ns)
    dx, _ = ns["gradient"](pos, q, a, b)
    assert np.max(np.abs(dx - fx)) > 1e-3 * np.max(np.abs(fx))


def test_dipole_direct_is_the_limit_of_charge_pairs():
    """A dipole against the charge pair +-|p|/e at x_j +- (e/2) p/|p| (the
    oracle's C direct sum), e -> 0."""
    rng = np.random.default_rng(5)
    pos = rng.random((30, 3))
    dip = rng.standard_normal((30, 3))
    psi, g = FG.dipole_direct(pos, dip)
    e = 1e-5
    for k in (0, 7):
        others = [j for j in range(30) if j != k]
        src = np.concatenate([pos[others] + 0.5 * e * dip[others], pos[others] - 0.5 * e * dip[others], pos[[k]]])
        qs = np.concatenate([np.full(29, 1.0 / e), np.full(29, -1.0 / e), [0.0]])
        phi, grad = O.direct_targets(src, qs, [58])
        assert abs(phi[0] - psi[k]) <= 1e-6 * max(1.0, abs(psi[k]))
        assert np.max(np.abs(grad[0] - g[k])) <= 1e-5 * max(1.0, np.max(np.abs(g[k])))


def test_gradient_from_one_charge_pass_and_dipole_passes():
    """The decomposition an FMM backward would run: dL/dq = phi^(a) + b . E +
    psi and dL/dx = a grad phi + q grad phi^(a) - q H b + q grad psi, with psi
    the potential of the dipoles -q_i b_i and the Hessian's columns the
    gradients of the potentials of the dipoles -q_j e_c."""
    pos, q, a, b = _system(80, 6)
    dx, dq = FG.gradient(pos, q, a, b)
    phi, g = O.direct(pos, q)
    pha, ga = O.direct(pos, a)
    psi, gpsi = FG.dipole_direct(pos, -q[:, None] * b)
    H = np.stack([FG.dipole_direct(pos, -q[:, None] * np.eye(3)[c][None, :])[1] for c in range(3)], axis=2)
    hb = np.einsum("kic,kc->ki", H, b)
    assert np.allclose(dq, pha - np.einsum("kc,kc->k", b, g) + psi, rtol=1e-12, atol=1e-12)
    assert np.allclose(dx, a[:, None] * g + q[:, None] * ga - q[:, None] * hb + q[:, None] * gpsi,
                       rtol=1e-12, atol=1e-12)


def test_dipole_multipole_is_the_limit_of_charge_pairs():
    """p2m_dipole against the P2M of the charge pair +-1/e at x +- (e/2) p."""
    rng = np.random.default_rng(8)
    c = np.array([0.5, 0.5, 0.5])
    pos = c + 0.1 * rng.standard_normal((5, 3))
    dip = rng.standard_normal((5, 3))
    for p in (1, 4, 7):
        M = FG.p2m_dipole(p, c, pos, dip)
        e = 1e-5
        pair = (O.p2m(p, c, pos + 0.5 * e * dip, np.full(5, 1.0 / e)) -
                O.p2m(p, c, pos - 0.5 * e * dip, np.full(5, 1.0 / e)))
        assert np.max(np.abs(M - pair)) <= 1e-6 * max(1.0, np.max(np.abs(M))), p


def test_dipole_multipole_far_field():
    """The dipoles' multipole, evaluated far away (M2P), converges in p to
    their direct potential."""
    rng = np.random.default_rng(9)
    c = np.array([0.5, 0.5, 0.5])
    pos = c + 0.05 * rng.standard_normal((8, 3))
    dip = rng.standard_normal((8, 3))
    y = np.array([1.4, -0.3, 0.9])
    allpos = np.vstack([pos, y])
    ref, _ = FG.dipole_direct(allpos, np.vstack([dip, np.zeros(3)]))
    err = [abs(O.m2p(p, FG.p2m_dipole(p, c, pos, dip), y - c) - ref[-1]) for p in (2, 4, 6, 8)]
    assert all(b < a / 5 for a, b in zip(err, err[1:])), err
    assert err[-1] <= 1e-7 * abs(ref[-1]), err


def test_dipole_fmm_and_fmm_gradient_converge():
    """The dipole-source FMM through the oracle tree's lists tends to the
    dipoles' direct sum (exactly equal with no M2L pair), and the FMM form of
    the force-loss gradient tends to the closed form."""
    import workloads as W
    wl = W.make_workload("plummer", n=600)
    rng = np.random.default_rng(3)
    a, b = rng.standard_normal(600), rng.standard_normal((600, 3))
    psi0, g0 = FG.dipole_direct(wl.pos, b)
    t0 = O.build_tree(wl.pos, 16, 1e-6)
    assert len(t0.m2l) == 0
    psi, g = FG.dipole_fmm(t0, wl.pos, b, 2)
    assert O.rel_l2(psi, psi0) <= 1e-12 and O.rel_l2(g, g0) <= 1e-12
    t = O.build_tree(wl.pos, 16, 0.5)
    e_psi, e_g = [], []
    for p in (2, 4, 6):
        psi, g = FG.dipole_fmm(t, wl.pos, b, p)
        e_psi.append(O.rel_l2(psi, psi0))
        e_g.append(O.rel_l2(g, g0))
    assert all(y < x / 2 for x, y in zip(e_psi, e_psi[1:])), e_psi
    assert all(y < x / 2 for x, y in zip(e_g, e_g[1:])), e_g
    dx0, dq0 = FG.gradient(wl.pos, wl.q, a, b)
    ex = [O.rel_l2(FG.fmm_gradient(t, wl.pos, wl.q, a, b, p)[0], dx0) for p in (2, 6)]
    assert ex[1] < ex[0] / 4 and ex[1] <= 2e-3, ex
