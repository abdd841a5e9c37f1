"""Batched trees: many independent systems in one tree and one evaluation."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.gpu_common import torch_dev

pytestmark = pytest.mark.gpu


def _systems(nsys, lo=300, hi=6000, seed=7):
    sizes = W.batched_sizes(nsys, lo=lo, hi=hi, seed=seed)
    systems = W.make_batched(nsys, seed=seed, sizes=sizes)
    pos = np.concatenate([s[0] for s in systems])
    q = np.concatenate([s[1] for s in systems])
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return systems, pos, q, off


def _batched(pos, off, **kw):
    import paper_1203_0889_gb300 as fmm
    torch, dev = torch_dev()
    return fmm.build_tree_batched(torch.tensor(pos, dtype=torch.float64, device=dev), off, **kw)


@pytest.mark.parametrize("leaf,theta", [(32, 0.5), (8, 0.4)])
def test_batched_tree_matches_oracle_per_system(leaf, theta):
    systems, pos, q, off = _systems(9)
    t = _batched(pos, off, p=2, leaf_size=leaf, theta=theta)
    ex = t.export()
    org, side, csys = t.export_systems()
    info = t.info()
    assert info.nsys == 9 and np.all(csys[:9] == np.arange(9))
    for s, (ps, _) in enumerate(systems):
        ref = O.build_tree(ps, leaf, theta)
        a, b = off[s], off[s + 1]
        assert np.array_equal(ex["keys"][a:b], ref.keys)
        assert np.array_equal(ex["perm"][a:b] - a, ref.perm)
        assert np.array_equal(org[s], ref.origin) and side[s] == ref.side
        cells = np.nonzero(csys == s)[0]
        local = -np.ones(info.ncell, np.int64)
        local[cells] = np.arange(len(cells))
        assert np.array_equal(ex["level"][cells], ref.level)
        assert np.array_equal(ex["cell_key"][cells], ref.cell_key)
        assert np.array_equal(ex["first"][cells] - a, ref.first)
        assert np.array_equal(ex["count"][cells], ref.count)
        par = ex["parent"][cells]
        assert np.array_equal(np.where(par >= 0, local[np.maximum(par, 0)], -1), ref.parent)
        assert np.array_equal(ex["child_count"][cells], ref.child_count)
        for name in ("m2l", "p2p"):
            lst = ex[name][np.isin(ex[name][:, 0], cells)]
            assert np.all(np.isin(lst[:, 1], cells))
            mapped = local[lst]
            mapped = mapped[np.lexsort((mapped[:, 1], mapped[:, 0]))]
            assert np.array_equal(mapped, getattr(ref, name))


@pytest.mark.parametrize("prec", [0, 2, 3])
def test_batched_values(prec):
    import paper_1203_0889_gb300 as fmm
    torch, dev = torch_dev()
    systems, pos, q, off = _systems(7)
    t = _batched(pos, off, p=6, leaf_size=32, theta=0.5, precision=prec)
    phi, f = t.evaluate(torch.tensor(q, dtype=torch.float64, device=dev))
    torch.cuda.synchronize()
    assert t.status() == fmm.FMM_OK
    phi, f = phi.cpu().numpy(), f.cpu().numpy()
    for s, (ps, qs) in enumerate(systems):
        a, b = off[s], off[s + 1]
        ref_phi, ref_g = O.fmm_evaluate(ps, qs, p=6, leaf_size=32, theta=0.5, nthreads=8)
        tol = 1e-10 if prec == 0 else 1e-4
        assert O.rel_l2(phi[a:b], ref_phi) <= tol
        assert O.rel_l2(f[a:b], -qs[:, None] * ref_g) <= tol
        # the same system alone, on its own tree, gives the same result
        if s < 3:
            ts = fmm.build_tree(torch.tensor(ps, dtype=torch.float64, device=dev), p=6, leaf_size=32, theta=0.5,
                                precision=prec)
            p1, f1 = ts.evaluate(torch.tensor(qs, dtype=torch.float64, device=dev))
            lim = 1e-13 if prec == 0 else 2e-5
            assert O.rel_l2(phi[a:b], p1.cpu().numpy()) <= lim


def test_batched_graph_replay():
    import paper_1203_0889_gb300 as fmm
    torch, dev = torch_dev()
    systems, pos, q, off = _systems(12)
    t = _batched(pos, off, p=6, leaf_size=32, theta=0.5, precision=2)
    qt = torch.tensor(q, dtype=torch.float32, device=dev)
    phi = torch.empty(len(q), dtype=torch.float32, device=dev)
    force = torch.empty((len(q), 3), dtype=torch.float32, device=dev)
    eager_phi, eager_f = t.evaluate(qt)
    g = fmm.capture_graph(t, qt, phi, force)
    phi.zero_(); force.zero_()
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    assert t.status() == fmm.FMM_OK
    assert torch.equal(phi, eager_phi) and torch.equal(force, eager_f)


def test_batched_argument_errors():
    import paper_1203_0889_gb300 as fmm
    torch, dev = torch_dev()
    pos = torch.rand((100, 3), dtype=torch.float64, device=dev)
    for off in ([0, 50, 50, 100], [1, 100], [0, 60, 40, 100]):
        with pytest.raises((fmm.FMMError, ValueError)):
            fmm.build_tree_batched(pos, off)


def test_autotuner_returns_a_candidate():
    import paper_1203_0889_gb300 as fmm
    torch, dev = torch_dev()
    systems, pos, q, off = _systems(16)
    best, times = fmm.autotune_leaf_size(torch.tensor(pos, dtype=torch.float64, device=dev),
                                         torch.tensor(q, dtype=torch.float32, device=dev), offsets=off,
                                         candidates=(16, 32, 64), repeats=1, p=6, theta=0.5, precision=2)
    assert best in (16, 32, 64) and all(v > 0 for v in times.values())


@pytest.mark.parametrize("leaf", [1, 16, 200])
def test_batched_octree_paths_agree(leaf):
    """The one-pass octree and the level-by-level one (FMM_BUILD_FALLBACKS)
    give the same batched tree and lists, with systems of one particle and
    systems below and above the leaf size (sizes 1 .. 1184)."""
    import paper_1203_0889_gb300 as fmm
    systems, pos, q, off = _systems(11, lo=1, hi=2500, seed=23)
    assert np.diff(off).min() == 1
    a = _batched(pos, off, p=2, leaf_size=leaf, theta=0.5).export()
    b = _batched(pos, off, p=2, leaf_size=leaf, theta=0.5, flags=fmm.BUILD_FALLBACKS).export()
    for k in a:
        assert np.array_equal(np.asarray(a[k]), np.asarray(b[k])), k
