"""The persistent task-queue evaluation: same results as the stage-by-stage
kernels, deterministic, and bounded waits that end in an error status."""
import time

import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.gpu_common import gpu_eval, gpu_tree, torch_dev

pytestmark = pytest.mark.gpu


# Precision 1 (FP32 P2P, FP64 expansions): the stage-by-stage kernel splits the
# near-field list of a leaf with many source records over several blocks and
# adds their FP32 partial sums in FP64, where the task queue sums the whole list
# in one FP32 stream, so the two differ by FP32 rounding of the near field.
@pytest.mark.parametrize("prec,tol", [(0, 1e-13), (1, 1e-6), (2, 1e-5)])
@pytest.mark.parametrize("name,n,p,leaf,theta", [("plummer", 30000, 8, 64, 0.4), ("clustered", 20000, 5, 16, 0.5),
                                                 ("uniform", 3000, 12, 32, 0.6)])
def test_queue_matches_staged(prec, tol, name, n, p, leaf, theta):
    import paper_1203_0889_gb300 as fmm
    wl = W.make_workload(name, n=n)
    tq = gpu_tree(wl.pos, p=p, leaf_size=leaf, theta=theta, precision=prec)
    ts = gpu_tree(wl.pos, p=p, leaf_size=leaf, theta=theta, precision=prec, flags=fmm.STAGED)
    pq, fq = gpu_eval(tq, wl.q)
    ps, fs = gpu_eval(ts, wl.q)
    assert tq.status() == fmm.FMM_OK and ts.status() == fmm.FMM_OK
    assert O.rel_l2(pq, ps) <= tol and O.rel_l2(fq, fs) <= tol


def test_queue_deterministic():
    torch, dev = torch_dev()
    wl = W.make_workload("plummer", n=40000)
    t = gpu_tree(wl.pos, p=6, leaf_size=32, theta=0.5, precision=2)
    q = torch.tensor(wl.q, dtype=torch.float64, device=dev)
    a = [t.evaluate(q) for _ in range(3)]
    torch.cuda.synchronize()
    for b in a[1:]:
        assert torch.equal(a[0][0], b[0]) and torch.equal(a[0][1], b[1])


@pytest.mark.parametrize("counter", [0, 1, 2, 3])
def test_queue_timeout_on_missing_dependency(counter):
    """A dependency counter raised by one on the host leaves a task never ready;
    the kernel's bounded waits end with FMM_ERR_TIMEOUT and the device stays usable."""
    import paper_1203_0889_gb300 as fmm
    torch, dev = torch_dev()
    wl = W.make_workload("uniform", n=20000)
    t = gpu_tree(wl.pos, p=4, leaf_size=32, theta=0.5, precision=2, timeout_ns=200_000_000)
    ex = t.export()
    leaf = int(np.nonzero(ex["child_count"] == 0)[0][-1])
    internal = int(np.nonzero(ex["child_count"] > 0)[0][-1])
    with_list = int(np.unique(ex["m2l"][:, 0])[-1])
    cell = {0: internal, 1: with_list, 2: leaf, 3: leaf}[counter]
    t.inject_dependency(counter, cell, 1)
    q = torch.tensor(wl.q, dtype=torch.float64, device=dev)
    t0 = time.time()
    t.evaluate(q)
    st = t.status()
    assert st == fmm.FMM_ERR_TIMEOUT
    assert time.time() - t0 < 30
    # the context still works: a fresh tree evaluates correctly
    t2 = gpu_tree(wl.pos, p=4, leaf_size=32, theta=0.5, precision=2)
    phi, f = gpu_eval(t2, wl.q)
    assert t2.status() == fmm.FMM_OK and np.all(np.isfinite(phi))
