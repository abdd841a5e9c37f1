"""Device octree and interaction lists against the oracle: bit-exact."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.gpu_common import assert_tree_equal, gpu_tree, torch_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["uniform", "plummer", "clustered"])
@pytest.mark.parametrize("n,leaf,theta", [(5000, 64, 0.5), (20000, 32, 0.4), (3000, 1, 0.7), (70000, 64, 0.4)])
def test_tree_bit_exact(name, n, leaf, theta):
    wl = W.make_workload(name, n=n)
    t = gpu_tree(wl.pos, p=2, leaf_size=leaf, theta=theta)
    assert_tree_equal(t.export(), O.build_tree(wl.pos, leaf, theta))


@pytest.mark.parametrize("name,n,leaf", [("uniform", 40000, 4096), ("clustered", 30000, 1000), ("plummer", 25000, 257)])
def test_tree_large_leaves(name, n, leaf):
    """Leaf sizes far above the usual: the one-pass octree's window of
    leaf + 1 particles spans many blocks of the level pass."""
    wl = W.make_workload(name, n=n)
    t = gpu_tree(wl.pos, p=2, leaf_size=leaf, theta=0.5)
    assert_tree_equal(t.export(), O.build_tree(wl.pos, leaf, 0.5))


def test_tree_fp32_positions():
    torch, _ = torch_dev()
    wl = W.make_workload("plummer", n=10000)
    p32 = wl.pos.astype(np.float32)
    t = gpu_tree(p32.astype(np.float64), p=2, leaf_size=16, theta=0.5, pos_dtype=torch.float32)
    assert_tree_equal(t.export(), O.build_tree(p32.astype(np.float64), 16, 0.5))


@pytest.mark.parametrize("case", ["one", "two", "coincident", "duplicates", "planar", "line", "tiny_leaf",
                                  "leaf_ge_n", "theta_small", "theta_large"])
def test_tree_edge_cases(case):
    rng = np.random.default_rng(11)
    leaf, theta = 8, 0.5
    if case == "one":
        pos = np.array([[0.1, 0.2, 0.3]])
    elif case == "two":
        pos = np.array([[0.0, 0.0, 0.0], [1.0, 1.0, 1.0]])
        leaf = 1
    elif case == "coincident":
        pos = np.tile([[0.5, -0.25, 3.0]], (100, 1))
    elif case == "duplicates":
        pos = rng.random((2000, 3)); pos[500:900] = pos[3]
    elif case == "planar":
        pos = np.c_[rng.random(3000), rng.random(3000), np.zeros(3000)]
    elif case == "line":
        pos = np.c_[rng.random(3000), np.full(3000, 2.0), np.full(3000, -1.0)]
    elif case == "tiny_leaf":
        pos = rng.random((4000, 3)); leaf = 1
    elif case == "leaf_ge_n":
        pos = rng.random((100, 3)); leaf = 100
    elif case == "theta_small":
        pos = rng.random((3000, 3)); theta = 1e-6
    else:
        pos = rng.random((3000, 3)); theta = 0.99
    t = gpu_tree(pos, p=2, leaf_size=leaf, theta=theta)
    assert_tree_equal(t.export(), O.build_tree(pos, leaf, theta))


def test_tree_empty():
    torch, dev = torch_dev()
    import paper_1203_0889_gb300 as fmm
    t = fmm.build_tree(torch.zeros((0, 3), dtype=torch.float64, device=dev), p=3)
    info = t.info()
    assert info.n == 0 and info.ncell == 0 and info.nm2l == 0 and info.np2p == 0
    phi, force = t.evaluate(torch.zeros(0, dtype=torch.float64, device=dev))
    assert phi.numel() == 0 and force.numel() == 0


def test_non_finite_positions_rejected():
    torch, dev = torch_dev()
    import paper_1203_0889_gb300 as fmm
    pos = torch.rand((100, 3), dtype=torch.float64, device=dev)
    pos[17, 1] = float("nan")
    with pytest.raises(fmm.FMMError) as e:
        fmm.build_tree(pos, p=3)
    assert e.value.code == fmm.FMM_ERR_ARG


@pytest.mark.parametrize("name,n,leaf,theta,prec", [("plummer", 60000, 32, 0.4, 3), ("clustered", 50000, 16, 0.5, 3),
                                                    ("uniform", 30000, 24, 0.5, 2)])
def test_build_fallback_paths_bit_exact(name, n, leaf, theta, prec):
    """FMM_BUILD_FALLBACKS builds the octree level by level (instead of in one
    pass) and forces the round-by-round traversal and (mixed mode) the
    sort-based class grouping, which otherwise run only on overflow: the tree
    and both lists still match the oracle bit for bit, and the class structure
    matches the default build."""
    import paper_1203_0889_gb300 as fmm
    wl = W.make_workload(name, n=n)
    ref = O.build_tree(wl.pos, leaf, theta)
    a = gpu_tree(wl.pos, p=6, leaf_size=leaf, theta=theta, precision=prec, flags=fmm.BUILD_FALLBACKS)
    b = gpu_tree(wl.pos, p=6, leaf_size=leaf, theta=theta, precision=prec)
    assert_tree_equal(a.export(), ref)
    assert_tree_equal(b.export(), ref)
    ia, ib = a.info(), b.info()
    assert (ia.tc_pairs, ia.tc_classes, ia.tc_items) == (ib.tc_pairs, ib.tc_classes, ib.tc_items)
