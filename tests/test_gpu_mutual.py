"""Mutual near-field interaction (FMM_MUTUAL, paper Section 4): the pairs of
two different leaves are evaluated once and added to both leaves.

The mutual form changes only the order and grouping of the FP32 P2P sums, so
it is held to the non-mutual form's bars against the oracle, and to the
non-mutual GPU result on the same tree within a few FP32 roundings.  The cases
cover every ring width (leaf sizes 1 .. 200, so target chunks of 1 .. 64 and a
second chunk), leaves split over several work items, the all-near-field limit
(theta -> 0, against the direct sum) and the batched tree."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.gpu_common import gpu_eval, gpu_tree, oracle_phi_force, torch_dev

pytestmark = pytest.mark.gpu

# the non-mutual form's measured-error bars (test_gpu_parity.py)
TIGHT = {1: 5e-6, 2: 1e-5, 3: 2e-5}
# mutual against non-mutual on one tree: the FP32 sums in another order and
# each cross-leaf separation rounded in one leaf's frame instead of both
SAME = 1e-6


def _flags(prec):
    import paper_1203_0889_gb300 as fmm
    return fmm.MUTUAL | (fmm.STAGED if prec != 3 else 0)


@pytest.mark.parametrize("prec", [1, 2, 3])
@pytest.mark.parametrize("name,n,p,leaf,theta", [
    ("uniform", 16384, 4, 64, 0.5),
    ("plummer", 30000, 8, 64, 0.4),
    ("clustered", 30000, 10, 64, 0.5),
])
def test_mutual_matches_oracle(prec, name, n, p, leaf, theta):
    import paper_1203_0889_gb300 as fmm
    wl = W.make_workload(name, n=n)
    ref_phi, ref_f, _ = oracle_phi_force(wl.pos, wl.q, p, leaf, theta)
    t = gpu_tree(wl.pos, p=p, leaf_size=leaf, theta=theta, precision=prec, flags=_flags(prec))
    phi, f = gpu_eval(t, wl.q)
    assert t.status() == fmm.FMM_OK
    e_phi, e_f = O.rel_l2(phi, ref_phi), O.rel_l2(f, ref_f)
    assert e_phi <= TIGHT[prec] and e_f <= TIGHT[prec], (e_phi, e_f)
    # the same tree without the mutual form
    t1 = gpu_tree(wl.pos, p=p, leaf_size=leaf, theta=theta, precision=prec,
                  flags=fmm.STAGED if prec != 3 else 0)
    phi1, f1 = gpu_eval(t1, wl.q)
    assert O.rel_l2(phi, phi1) <= SAME and O.rel_l2(f, f1) <= SAME


@pytest.mark.parametrize("leaf,n", [(1, 2500), (3, 4000), (8, 6000), (33, 6000), (64, 8000), (100, 8000),
                                    (200, 9000)])
def test_mutual_near_field_only_equals_direct(leaf, n):
    """theta -> 0: no M2L, every leaf pair is near; the mutual FP32 near field
    against the FP64 direct sum (leaf sizes from one particle to two target
    chunks of 64 and more)."""
    import paper_1203_0889_gb300 as fmm
    wl = W.make_workload("plummer", n=n)
    ref_phi, ref_grad = O.direct(wl.pos, wl.q)
    t = gpu_tree(wl.pos, p=2, leaf_size=leaf, theta=1e-6, precision=fmm.PREC_FP32_P2P,
                 flags=fmm.MUTUAL | fmm.STAGED)
    assert t.info().nm2l == 0
    phi, f = gpu_eval(t, wl.q)
    assert t.status() == fmm.FMM_OK
    assert O.rel_l2(phi, ref_phi) <= 2e-6
    assert O.rel_l2(f, -wl.q[:, None] * ref_grad) <= 2e-6


@pytest.mark.parametrize("R", [8, 16, 256])
def test_mutual_split_items(R):
    """Leaves split over work items of R records (8 is the smallest the library
    takes) give the same result as whole leaves."""
    import paper_1203_0889_gb300 as fmm
    torch, dev = torch_dev()
    wl = W.make_workload("clustered", n=40000)
    pos = torch.tensor(wl.pos, dtype=torch.float64, device=dev)
    q = torch.tensor(wl.q, dtype=torch.float32, device=dev)
    kw = dict(p=8, leaf_size=32, theta=0.5, precision=fmm.PREC_MIXED_TC)
    a = fmm.build_tree(pos, flags=fmm.MUTUAL, p2p_item_records=R, **kw)
    b = fmm.build_tree(pos, **kw)
    pa, fa = a.evaluate(q)
    pb, fb = b.evaluate(q)
    assert a.status() == fmm.FMM_OK
    assert ((pa - pb).norm() / pb.norm()).item() <= SAME
    assert ((fa - fb).norm() / fb.norm()).item() <= SAME


def test_mutual_repeat_and_fp64_ignored():
    """Repeated mutual evaluations agree to FP32 rounding (the atomics' order
    varies); with FMM_PREC_FP64 the flag changes nothing, bit for bit."""
    import paper_1203_0889_gb300 as fmm
    torch, dev = torch_dev()
    wl = W.make_workload("uniform", n=20000)
    pos = torch.tensor(wl.pos, dtype=torch.float64, device=dev)
    q = torch.tensor(wl.q, dtype=torch.float64, device=dev)
    t = fmm.build_tree(pos, p=6, leaf_size=32, theta=0.5, precision=fmm.PREC_FP32, flags=fmm.MUTUAL)
    a = t.evaluate(q)
    b = t.evaluate(q)
    assert ((a[0] - b[0]).norm() / a[0].norm()).item() <= 1e-7
    assert ((a[1] - b[1]).norm() / a[1].norm()).item() <= 1e-7
    c = fmm.build_tree(pos, p=6, leaf_size=32, theta=0.5, precision=fmm.PREC_FP64, flags=fmm.MUTUAL).evaluate(q)
    d = fmm.build_tree(pos, p=6, leaf_size=32, theta=0.5, precision=fmm.PREC_FP64).evaluate(q)
    assert torch.equal(c[0], d[0]) and torch.equal(c[1], d[1])


@pytest.mark.parametrize("prec", [1, 3])
def test_mutual_close_pair_within_a_leaf(prec):
    """The pairs within a leaf stay with the own-leaf kernel (separations from
    the coordinates' residuals) in the mutual form too."""
    import paper_1203_0889_gb300 as fmm
    rng = np.random.default_rng(7)
    pos = rng.random((6000, 3))
    pos[1] = pos[0] + np.array([1e-6, 0.0, 0.0])
    q = rng.uniform(-1, 1, 6000)
    t64 = gpu_tree(pos, p=6, leaf_size=32, theta=0.5, precision=fmm.PREC_FP64)
    t = gpu_tree(pos, p=6, leaf_size=32, theta=0.5, precision=prec, flags=_flags(prec))
    _, f64 = gpu_eval(t64, q)
    _, f = gpu_eval(t, q)
    for i in (0, 1):
        assert np.linalg.norm(f[i] - f64[i]) <= 1e-5 * np.linalg.norm(f64[i]), (i, f[i], f64[i])
    assert O.rel_l2(f, f64) <= 1e-5


def test_mutual_batched():
    """Several systems in one tree: the mutual form per system against the
    non-mutual form on the same batched tree."""
    import paper_1203_0889_gb300 as fmm
    torch, dev = torch_dev()
    systems = W.make_batched(12)
    sizes = np.array([len(s[1]) for s in systems], np.int64)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    pos = torch.tensor(np.concatenate([s[0] for s in systems]), dtype=torch.float64, device=dev)
    q = torch.tensor(np.concatenate([s[1] for s in systems]), dtype=torch.float32, device=dev)
    prm = dict(p=6, leaf_size=64, theta=0.5, precision=fmm.PREC_MIXED_TC)
    a = fmm.build_tree_batched(pos, off, flags=fmm.MUTUAL, **prm)
    b = fmm.build_tree_batched(pos, off, **prm)
    pa, fa = a.evaluate(q)
    pb, fb = b.evaluate(q)
    assert a.status() == fmm.FMM_OK
    pa, fa, pb, fb = (x.double().cpu().numpy() for x in (pa, fa, pb, fb))
    for s in range(len(systems)):
        sl = slice(off[s], off[s + 1])
        assert O.rel_l2(pa[sl], pb[sl]) <= SAME and O.rel_l2(fa[sl], fb[sl]) <= SAME, s
