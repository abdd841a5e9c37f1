"""Parity at full size, in the configuration bench.py times.

The 1M-particle Plummer workload (p = 8, leaf 64, theta = 0.4): the device tree
and lists are compared with the oracle's bit for bit, and the potentials and
forces of sampled leaves are compared with the oracle's FMM computed leaf by
leaf.  The 4M-particle clustered set checks the tree at the largest size."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.gpu_common import assert_tree_equal, torch_dev

pytestmark = pytest.mark.gpu

P, LEAF, THETA = 8, 64, 0.4


@pytest.fixture(scope="module")
def plummer():
    wl = W.make_workload("plummer")
    ref = O.build_tree(wl.pos, LEAF, THETA)
    leaves = np.nonzero(ref.is_leaf)[0]
    rng = np.random.default_rng(2026)
    samp = list(rng.choice(leaves, 24, replace=False))
    samp.append(int(leaves[np.argmax(ref.count[leaves])]))         # the fullest leaf
    samp.append(int(leaves[np.argmax(ref.level[leaves])]))         # the deepest leaf
    samp.append(int(leaves[np.argmin(ref.level[leaves])]))         # the shallowest leaf
    samp = np.array(sorted(set(samp)), np.int32)
    idx, phi, g = ref.evaluate_leaves(P, wl.q, samp)
    return wl, ref, idx, phi, -wl.q[idx, None] * g


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-4), (2, 1e-4), (3, 1e-4)])
def test_bench_workload(plummer, prec, tol):
    import paper_1203_0889_gb300 as fmm
    torch, dev = torch_dev()
    wl, ref, idx, ref_phi, ref_f = plummer
    pos = torch.tensor(wl.pos, dtype=torch.float64, device=dev)
    q = torch.tensor(wl.q, dtype=torch.float64, device=dev)
    t = fmm.build_tree(pos, p=P, leaf_size=LEAF, theta=THETA, precision=prec, flags=fmm.TIMING)
    if prec == 3:
        assert_tree_equal(t.export(), ref)
    phi, force = t.evaluate(q)
    torch.cuda.synchronize()
    assert t.status() == fmm.FMM_OK
    # stage timing: every build stage and the list sub-stages (nested in "lists")
    ms = t.stage_times()
    for name in ("keys", "octree", "setup", "lists", "traversal", "classes", "p2p_list", "prepare"):
        assert name in ms and ms[name] >= 0.0, name
    assert ("queue" in ms) != ("l2p" in ms)      # task-queue or stage-by-stage evaluation
    for name in ("traversal", "classes", "p2p_list"):
        assert ms[name] <= ms["lists"] + 1e-3, name
    phi, force = phi.cpu().numpy()[idx], force.cpu().numpy()[idx]
    assert O.rel_l2(phi, ref_phi) <= tol
    assert O.rel_l2(force, ref_f) <= tol


def test_largest_tree_bit_exact():
    import paper_1203_0889_gb300 as fmm
    torch, dev = torch_dev()
    wl = W.make_workload("clustered")
    t = fmm.build_tree(torch.tensor(wl.pos, dtype=torch.float64, device=dev), p=2, leaf_size=64, theta=0.5)
    assert_tree_equal(t.export(), O.build_tree(wl.pos, 64, 0.5))
