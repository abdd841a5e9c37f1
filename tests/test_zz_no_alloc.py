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


def _existing(pos_t, q_t, flags=0):
    import paper_1203_0889_gb300 as fmm
    # theta tiny: no pair is accepted for M2L, so the FMM is all P2P (the direct sum)
    t = fmm.build_tree(pos_t, p=2, leaf_size=64, theta=1e-6, precision=fmm.PREC_FP64, flags=flags)
    assert t.info().nm2l == 0
    phi, force = t.evaluate(q_t)
    return phi, force


def _noalloc(lib, pos_t, q_t, flags=0, want_phi=True, want_force=True):
    import torch
    n = q_t.shape[0]
    phi = torch.full((n,), float("nan"), dtype=q_t.dtype, device=q_t.device)
    force = torch.full((n, 3), float("nan"), dtype=q_t.dtype, device=q_t.device)
    code = 0 if q_t.dtype == torch.float64 else 1
    rc = lib.fmm_direct_noalloc(n, C.c_void_p(pos_t.data_ptr()), C.c_void_p(q_t.data_ptr()),
                                C.c_void_p(phi.data_ptr()) if want_phi else None,
                                C.c_void_p(force.data_ptr()) if want_force else None, code, flags,
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


def test_noalloc_fp32_field_and_missing_outputs():
    """The FP32 form (accumulated in FP64, rounded once: FP32 rounding of the
    result), the field instead of the force, and either output left out."""
    import torch

    import paper_1203_0889_gb300 as fmm
    lib = fmm.load()
    dev = torch.device("cuda:0")
    wl = W.make_workload("uniform", n=3000)
    pos = torch.tensor(wl.pos, dtype=torch.float64, device=dev)
    q = torch.tensor(wl.q, dtype=torch.float64, device=dev)
    ref_phi, ref_force = _existing(pos, q)
    # FP32: against the FP64 sum of the same FP32-rounded inputs; the one
    # difference left is the rounding of each result to FP32 (2^-24 relative)
    pos32, q32 = pos.float(), q.float()
    ref_phi32, ref_force32 = _existing(pos32.double(), q32.double())
    phi32, force32 = _noalloc(lib, pos32, q32)
    assert _rel(phi32.double(), ref_phi32) <= 1e-7 and _rel(force32.double(), ref_force32) <= 1e-7
    ref_phi_f, ref_field = _existing(pos, q, flags=fmm.OUT_FIELD)
    _, field = _noalloc(lib, pos, q, flags=fmm.OUT_FIELD)
    assert _rel(field, ref_field) <= TOL
    phi_only, untouched = _noalloc(lib, pos, q, want_force=False)
    assert _rel(phi_only, ref_phi) <= TOL and bool(torch.isnan(untouched).all())
    untouched, force_only = _noalloc(lib, pos, q, want_phi=False)
    assert _rel(force_only, ref_force) <= TOL and bool(torch.isnan(untouched).all())
