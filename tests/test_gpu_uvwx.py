"""The parent-neighbour-child list builder on the GPU (FMM_LISTS_UVWX; paper
Section 2.1, after Cheng, Greengard and Rokhlin 1999) against the oracle's
lists and values built from their definitions (oracle/uvwx.py, W and X as
direct sums): the M2L and P2P pairs exactly, the FP64 path within 1e-10 of the
oracle's FMM through the same lists, the reduced-precision paths within their
stated 1e-4 bar."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle import uvwx
from tests.gpu_common import gpu_eval, gpu_tree

pytestmark = pytest.mark.gpu

CASES = [("uniform", 1500, 16), ("plummer", 1500, 8), ("clustered", 2000, 16)]


@pytest.mark.parametrize("name,n,leaf", CASES)
def test_lists_match_oracle(name, n, leaf):
    import paper_1203_0889_gb300 as fmm
    wl = W.make_workload(name, n=n)
    ref = O.build_tree(wl.pos, leaf, 0.5)
    t = gpu_tree(wl.pos, p=4, leaf_size=leaf, theta=0.5, precision=fmm.PREC_FP64, flags=fmm.LISTS_UVWX)
    ex = t.export()
    m2l, p2p = uvwx.pair_lists(ref)
    assert np.array_equal(ex["keys"], ref.keys) and np.array_equal(ex["cell_key"], ref.cell_key)
    assert np.array_equal(ex["m2l"], m2l)
    assert np.array_equal(ex["p2p"], p2p)


@pytest.mark.parametrize("name,n,leaf,p", [("plummer", 1500, 8, 6), ("clustered", 2000, 16, 8)])
def test_fp64_matches_oracle(name, n, leaf, p):
    import paper_1203_0889_gb300 as fmm
    wl = W.make_workload(name, n=n)
    ref = O.build_tree(wl.pos, leaf, 0.5)
    phi_o, g_o = uvwx.evaluate(wl.pos, wl.q, p, tree=ref, wx="direct")
    t = gpu_tree(wl.pos, p=p, leaf_size=leaf, theta=0.5, precision=fmm.PREC_FP64, flags=fmm.LISTS_UVWX)
    phi, f = gpu_eval(t, wl.q)
    assert t.status() == fmm.FMM_OK
    assert O.rel_l2(phi, phi_o) <= 1e-10
    assert O.rel_l2(f, -wl.q[:, None] * g_o) <= 1e-10


@pytest.mark.parametrize("prec", [1, 2, 3])
def test_reduced_precision_within_bar(prec):
    import paper_1203_0889_gb300 as fmm
    wl = W.make_workload("plummer", n=1500)
    ref = O.build_tree(wl.pos, 8, 0.5)
    phi_o, g_o = uvwx.evaluate(wl.pos, wl.q, 8, tree=ref, wx="direct")
    t = gpu_tree(wl.pos, p=8, leaf_size=8, theta=0.5, precision=prec, flags=fmm.LISTS_UVWX)
    phi, f = gpu_eval(t, wl.q)
    assert t.status() == fmm.FMM_OK
    assert O.rel_l2(phi, phi_o) <= 1e-4 and O.rel_l2(f, -wl.q[:, None] * g_o) <= 1e-4
