"""Differentiable FMM: FMMFunction's backward against the direct-sum gradient
and against finite differences taken with the tree held fixed."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.gpu_common import torch_dev

pytestmark = pytest.mark.gpu


def _setup(n, p, prec, dtype=None, theta=0.5):
    import paper_1203_0889_gb300 as fmm
    torch, dev = torch_dev()
    dtype = dtype or torch.float64
    wl = W.make_workload("gradient", n=n)
    pos = torch.tensor(wl.pos, dtype=torch.float64, device=dev)
    q = torch.tensor(wl.q, dtype=dtype, device=dev)
    w = torch.tensor(wl.extra["w"], dtype=dtype, device=dev)
    tree = fmm.build_tree(pos, p=p, leaf_size=64, theta=theta, precision=prec, flags=fmm.OUT_FIELD)
    return fmm, torch, wl, pos, q, w, tree


def _grads(fmm, torch, pos, q, w, tree):
    posv = pos.clone().to(q.dtype).requires_grad_(True)
    qv = q.clone().requires_grad_(True)
    phi = fmm.FMMFunction.apply(posv, qv, tree)
    loss = (w * phi).sum()
    loss.backward()
    return phi.detach(), posv.grad.double().cpu().numpy(), qv.grad.double().cpu().numpy()


def test_backward_matches_direct_gradient():
    fmm, torch, wl, pos, q, w, tree = _setup(4096, 8, 0)
    phi, dx, dq = _grads(fmm, torch, pos, q, w, tree)
    wn = wl.extra["w"]
    phi_w, g_w = O.direct(wl.pos, wn)
    _, g_q = O.direct(wl.pos, wl.q)
    ref_dq = phi_w
    ref_dx = wn[:, None] * g_q + wl.q[:, None] * g_w
    assert O.rel_l2(dq, ref_dq) <= 1e-4
    assert O.rel_l2(dx, ref_dx) <= 1e-4


def test_backward_matches_finite_differences_fixed_tree():
    fmm, torch, wl, pos, q, w, tree = _setup(4096, 16, 0)
    phi, dx, dq = _grads(fmm, torch, pos, q, w, tree)
    h = 1e-6 * float(tree.info().side)

    def loss(x):
        tree.set_positions(x)
        ph, _ = tree.evaluate(q)
        return float((w * ph).sum().item())

    scale = np.abs(dx).max()
    for j in (0, 1000, 4095):
        for d in range(3):
            xp, xm = pos.clone(), pos.clone()
            xp[j, d] += h
            xm[j, d] -= h
            fd = (loss(xp) - loss(xm)) / (2 * h)
            assert abs(fd - dx[j, d]) <= 1e-6 * scale, (j, d, fd, dx[j, d])
    tree.set_positions(pos)
    # dq is exactly the potential of the weights on the same tree
    phw, _ = tree.evaluate(w)
    assert np.allclose(phw.cpu().numpy(), dq, rtol=0, atol=1e-12 * np.abs(dq).max())


@pytest.mark.parametrize("prec", [2, 3])
def test_reduced_precision_gradients(prec):
    fmm, torch, wl, pos, q, w, t64 = _setup(30000, 8, 0)
    _, dx64, dq64 = _grads(fmm, torch, pos, q, w, t64)
    _, torch_, _, pos, q32, w32, t32 = _setup(30000, 8, prec, dtype=torch.float32)
    _, dx32, dq32 = _grads(fmm, torch, pos, q32, w32, t32)
    assert O.rel_l2(dq32, dq64) <= 1e-4 and O.rel_l2(dx32, dx64) <= 1e-4


def test_backward_needs_field_tree():
    import paper_1203_0889_gb300 as fmm
    torch, dev = torch_dev()
    wl = W.make_workload("uniform", n=1000)
    pos = torch.tensor(wl.pos, dtype=torch.float64, device=dev)
    q = torch.tensor(wl.q, dtype=torch.float64, device=dev)
    t = fmm.build_tree(pos, p=4)
    with pytest.raises(ValueError):
        fmm.FMMFunction.apply(pos, q, t)
    with pytest.raises(fmm.FMMError) as e:
        t.backward(q, q, torch.zeros((1000, 3), dtype=torch.float64, device=dev))
    assert e.value.code == fmm.FMM_ERR_STATE


def test_function_follows_its_positions():
    """FMMFunction evaluates at the positions it is given: a tensor other than the
    tree's own (here the particles moved by a small shift) is loaded into the
    fixed tree first; a tensor of the wrong shape is refused."""
    fmm, torch, wl, pos, q, w, tree = _setup(4096, 8, 0)
    moved = pos + 1e-4 * float(tree.info().side)
    phi = fmm.FMMFunction.apply(moved.clone().requires_grad_(True), q, tree)
    ref = fmm.build_tree(pos, p=8, leaf_size=64, theta=0.5, precision=0, flags=fmm.OUT_FIELD)
    ref.set_positions(moved)
    phi_ref, _ = ref.evaluate(q)
    assert torch.equal(phi.detach(), phi_ref)
    # back at the tree's own positions: the same values as a plain evaluation
    phi0 = fmm.FMMFunction.apply(pos.clone().requires_grad_(True), q, tree)
    ref.set_positions(pos)
    assert torch.equal(phi0.detach(), ref.evaluate(q)[0])
    with pytest.raises(ValueError):
        fmm.FMMFunction.apply(pos[:100], q, tree)
