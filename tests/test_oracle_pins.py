"""The CPU oracle against closed forms, exact identities, bounds and brute force."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests import oracle_pins as P


@pytest.mark.parametrize("pin", [
    P.pin_direct_two_charges, P.pin_direct_cube_corners, P.pin_direct_coincident_and_third_law,
    P.pin_multipole_single_charge, P.pin_multipole_on_axis, P.pin_m2m_exact, P.pin_l2l_exact,
    P.pin_m2l_single_charge, P.pin_m2l_order_zero, P.pin_l2p_gradient_fd,
    P.pin_scaling_invariance, P.pin_fmm_equals_direct_without_far_field,
    P.pin_fmm_error_decays_with_p, P.pin_fmm_high_order_matches_direct, P.pin_fmm_net_force,
    P.pin_fmm_sampled_matches_full, P.pin_direct_gradient_formulas, P.pin_fmm_gradient_fixed_tree,
    P.pin_root_cube_centred, P.pin_traversal_tie_break,
], ids=lambda f: f.__name__)
def test_pin(pin):
    pin()


@pytest.mark.parametrize("name", ["uniform", "plummer", "clustered"])
@pytest.mark.parametrize("leaf,theta", [(16, 0.5), (8, 0.4), (1, 0.7)])
def test_tree_invariants(name, leaf, theta):
    P.pin_tree_invariants(W.make_workload(name, n=1500).pos, leaf, theta)


@pytest.mark.parametrize("name", ["uniform", "plummer", "clustered"])
@pytest.mark.parametrize("leaf,theta", [(16, 0.5), (4, 0.4), (32, 0.8)])
def test_lists_cover_every_pair_once(name, leaf, theta):
    P.pin_lists_cover_every_pair_once(W.make_workload(name, n=1200).pos, leaf, theta)


def test_degenerate_inputs():
    # empty input
    T = O.build_tree(np.zeros((0, 3)), 16, 0.5)
    assert T.ncell == 0 and len(T.m2l) == 0 and len(T.p2p) == 0
    # one particle: a root leaf that interacts with itself only, no result
    f, g = O.fmm_evaluate(np.array([[0.3, 0.2, 0.1]]), np.array([1.0]), p=4)
    assert f[0] == 0.0 and np.all(g == 0.0)
    # all particles on one point: one level-21 leaf holding them all, r = 0 skipped
    pos = np.tile([[0.5, 0.5, 0.5]], (40, 1))
    T = P.pin_tree_invariants(pos, 4, 0.5)
    assert T.child_count[T.ncell - 1] == 0 and T.level[T.ncell - 1] == 21
    f, g = T.evaluate(3, np.ones(40))
    assert np.all(f == 0.0) and np.all(g == 0.0)
    # duplicates mixed with distinct points still match the direct sum
    rng = np.random.default_rng(0)
    pos = rng.random((300, 3))
    pos[100:120] = pos[5]
    q = rng.uniform(-1, 1, 300)
    pd, gd = O.direct(pos, q)
    f, g = O.fmm_evaluate(pos, q, p=12, leaf_size=8, theta=0.4)
    assert O.rel_l2(f, pd) < 1e-4 and O.rel_l2(g, gd) < 1e-4


def test_planar_and_collinear():
    # all particles on a plane or a line: bounding box flat in some axes
    rng = np.random.default_rng(3)
    for pos in (np.c_[rng.random(500), rng.random(500), np.zeros(500)],
                np.c_[rng.random(500), np.full(500, 2.0), np.full(500, -1.0)]):
        q = rng.uniform(-1, 1, 500)
        P.pin_tree_invariants(pos, 8, 0.5)
        P.pin_lists_cover_every_pair_once(pos, 8, 0.5)
        pd, gd = O.direct(pos, q)
        f, g = O.fmm_evaluate(pos, q, p=10, leaf_size=8, theta=0.5)
        assert O.rel_l2(f, pd) < 1e-5


def test_threads_do_not_change_results():
    wl = W.make_workload("plummer", n=5000)
    T = O.build_tree(wl.pos, 32, 0.4)
    f1, g1 = T.evaluate(6, wl.q, nthreads=1)
    f4, g4 = T.evaluate(6, wl.q, nthreads=4)
    assert np.array_equal(f1, f4) and np.array_equal(g1, g4)


@pytest.mark.parametrize("name", ["uniform", "plummer", "clustered"])
@pytest.mark.parametrize("leaf,theta", [(8, 0.5), (1, 0.4), (32, 0.7)])
def test_split_rule_invariants(name, leaf, theta):
    P.pin_split_rule_invariants(W.make_workload(name, n=2000).pos, leaf, theta)
