"""The allocation-free direct evaluation against the existing entry points.

fmm_direct_noalloc serves callers that cannot allocate device memory (a
plug-in whose host framework owns all device memory, a real-time loop that
must not wait on the allocator); it keeps its scratch in a static device
array of the library.  This file is collected last so that a failure here
comes after every other test has run.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-10  # the FP64 parity tolerance of the other GPU tests


def _existing(pos_t, q_t):
    import paper_1203_0889_gb300 as fmm
    # theta tiny: no pair is accepted for M2L, so the FMM is all P2P (the direct sum)
    t = fmm.build_tree(pos_t, p=2, leaf_size=64, theta=1e-6, precision=fmm.PREC_FP64)
    assert t.info().nm2l == 0
    phi, force = t.evaluate(q_t)
    return phi, force


def _noalloc(lib, pos_t, q_t):
    import torch
    n = q_t.shape[0]
    phi = torch.full((n,), float("nan"), dtype=q_t.dtype, device=q_t.device)
    force = torch.full((n, 3), float("nan"), dtype=q_t.dtype, device=q_t.device)
    rc = lib.fmm_direct_noalloc(n, C.c_void_p(pos_t.data_ptr()), C.c_void_p(q_t.data_ptr()),
                                C.c_void_p(phi.data_ptr()), C.c_void_p(force.data_ptr()), 0, 0,
                                C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, lib.fmm_last_error()
    return phi, force


def _rel(a, b):
    return float((a - b).norm() / b.norm())


def test_noalloc_matches_existing_entry_point_on_two_calls():
    import torch

    import paper_1203_0889_gb300 as fmm
    lib = fmm.load()
    dev = torch.device("cuda:0")
    nmax = int(lib.fmm_direct_noalloc_max_n())
    assert nmax == 16384
    # call 1 fills the whole scratch; call 2 is a smaller system, so stale
    # records of call 1 sit beyond its end and its accumulators must be cleared
    for name, n in (("plummer", nmax), ("clustered", 5000)):
        wl = W.make_workload(name, n=n)
        pos = torch.tensor(wl.pos, dtype=torch.float64, device=dev)
        q = torch.tensor(wl.q, dtype=torch.float64, device=dev)
        phi, force = _noalloc(lib, pos, q)
        ref_phi, ref_force = _existing(pos, q)
        torch.cuda.synchronize()
        assert _rel(phi, ref_phi) <= TOL and _rel(force, ref_force) <= TOL


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch

    import paper_1203_0889_gb300 as fmm
    lib = fmm.load()
    n = int(lib.fmm_direct_noalloc_max_n()) + 1
    rc = lib.fmm_direct_noalloc(n, C.c_void_p(16), C.c_void_p(16), None, None, 0, 0, None)
    assert rc == fmm.FMM_ERR_ARG
    assert b"static scratch" in lib.fmm_last_error()
