"""Helpers shared by the GPU tests (inputs from workloads, references from the oracle)."""
import numpy as np

import oracle as O

TREE_KEYS = ("keys", "perm", "level", "cell_key", "first", "count", "parent", "child_first", "child_count",
             "m2l", "p2p")


def torch_dev():
    import torch
    return torch, torch.device("cuda:0")


def gpu_tree(pos, **kw):
    import paper_1203_0889_gb300 as fmm
    torch, dev = torch_dev()
    t = torch.tensor(pos, dtype=kw.pop("pos_dtype", torch.float64), device=dev)
    return fmm.build_tree(t, **kw)


def assert_tree_equal(ex, ref):
    for k in TREE_KEYS:
        a, b = ex[k], getattr(ref, k)
        assert a.shape == b.shape, (k, a.shape, b.shape)
        assert np.array_equal(a, b), (k, np.argwhere(a != b)[:5])
    assert np.array_equal(ex["origin"], ref.origin) and ex["side"] == ref.side


def gpu_eval(tree, q, dtype=None):
    torch, dev = torch_dev()
    dtype = dtype or torch.float64
    qt = torch.tensor(q, dtype=dtype, device=dev)
    phi, force = tree.evaluate(qt)
    torch.cuda.synchronize()
    return phi.double().cpu().numpy(), force.double().cpu().numpy()


def oracle_phi_force(pos, q, p, leaf, theta):
    T = O.build_tree(pos, leaf, theta)
    phi, grad = T.evaluate(p, q, nthreads=8)
    return phi, -q[:, None] * grad, T
