"""GB300 (sm_103a) adaptive 3-D Laplace FMM -- Python binding of the C ABI.

This module only marshals arguments: every step of the tree build and the
evaluation runs in the CUDA library ``libfmm_gb300.so`` (declared in
``include/fmm.h``).  PyTorch provides device memory and streams.  There is no
CPU fallback: without the compiled library every call raises.

    tree = build_tree(pos, p=8, leaf_size=64, theta=0.4, precision=PREC_FP32_P2P)
    phi, force = tree.evaluate(q)

The method is the one of "Data-Driven Execution of Fast Multipole Methods"
(Ltaief & Yokota): adaptive octree (Section 2.1), Morton keys (Section 2.2),
breadth-first dual tree traversal (Sections 4, 5), P2M/M2M/M2L/L2L/L2P/P2P
(Section 2.1), non-mutual target-owned interaction (Section 4).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

__all__ = [
    "FMM_OK", "FMM_ERR_ARG", "FMM_ERR_ALLOC", "FMM_ERR_CUDA", "FMM_ERR_TIMEOUT", "FMM_ERR_STATE",
    "PREC_FP64", "PREC_FP32_P2P", "PREC_FP32", "PREC_MIXED_TC", "OUT_FIELD", "STAGED", "TIMING", "NO_OVERLAP", "BUILD_FALLBACKS",
    "TASK_GRAPH", "MUTUAL", "LISTS_UVWX",
    "FMMError", "Params", "TreeInfo", "Tree", "build_tree", "build_tree_batched", "evaluate", "library_path", "load",
    "capture_graph", "autotune_leaf_size", "autotune",
]

FMM_OK, FMM_ERR_ARG, FMM_ERR_ALLOC, FMM_ERR_CUDA, FMM_ERR_TIMEOUT, FMM_ERR_STATE = 0, -1, -2, -3, -4, -5
F64, F32 = 0, 1
PREC_FP64, PREC_FP32_P2P, PREC_FP32, PREC_MIXED_TC = 0, 1, 2, 3
OUT_FIELD, STAGED, TIMING, NO_OVERLAP, BUILD_FALLBACKS, TASK_GRAPH, MUTUAL, LISTS_UVWX = 1, 2, 4, 8, 16, 32, 64, 128
STAGE_NAMES = ("keys", "octree", "lists", "setup", "prepare", "p2p", "p2m", "m2m", "m2l", "l2l", "l2p", "queue",
               "m2l_tc", "traversal", "classes", "p2p_list")

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libfmm_gb300.so")
_lib = None
_lock = threading.Lock()


class FMMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class Params(C.Structure):
    _fields_ = [("p", C.c_int32), ("leaf_size", C.c_int32), ("theta", C.c_double),
                ("precision", C.c_int32), ("flags", C.c_int32), ("timeout_ns", C.c_int64),
                ("p2p_item_records", C.c_int32), ("tc_min_pairs", C.c_int32)]


class TreeInfo(C.Structure):
    _fields_ = [("n", C.c_int64), ("ncell", C.c_int32), ("nlevel", C.c_int32), ("nleaf", C.c_int32),
                ("p", C.c_int32), ("nm2l", C.c_int64), ("np2p", C.c_int64), ("origin", C.c_double * 3),
                ("side", C.c_double), ("device_bytes", C.c_int64), ("tc_pairs", C.c_int64),
                ("tc_classes", C.c_int64), ("tc_items", C.c_int64), ("nsys", C.c_int64)]


def library_path() -> str:
    return _LIB_PATH


_P = C.c_void_p


def load():
    """Load the compiled library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_LIB_PATH):
                raise ImportError(f"{_LIB_PATH} is missing: build it with "
                                  "`python -c 'import __graft_entry__ as g; g.build()'`")
            lib = C.CDLL(_LIB_PATH)
            lib.fmm_build_tree.argtypes = [C.POINTER(Params), C.c_int64, _P, C.c_int, C.POINTER(_P), _P]
            lib.fmm_evaluate.argtypes = [_P, _P, _P, _P, C.c_int, _P]
            lib.fmm_build_tree_batched.argtypes = [C.POINTER(Params), C.c_int32, _P, _P, C.c_int,
                                                   C.POINTER(_P), _P]
            lib.fmm_evaluate_batched.argtypes = [_P, _P, _P, _P, C.c_int, _P]
            lib.fmm_tree_get_info.argtypes = [_P, C.POINTER(TreeInfo)]
            lib.fmm_tree_export.argtypes = [_P] + [_P] * 11
            lib.fmm_status.argtypes = [_P]
            lib.fmm_tree_destroy.argtypes = [_P]
            lib.fmm_tree_destroy.restype = None
            lib.fmm_last_error.restype = C.c_char_p
            lib.fmm_version.restype = C.c_char_p
            lib.fmm_stage_times.argtypes = [_P, _P, C.c_int32]
            lib.fmm_stage_times.restype = C.c_int
            lib.fmm_stage_name.argtypes = [C.c_int32]
            lib.fmm_stage_name.restype = C.c_char_p
            lib.fmm_kernel_launches.argtypes = [_P, C.c_int32]
            lib.fmm_kernel_launches.restype = C.c_int64
            lib.fmm_tree_export_systems.argtypes = [_P, _P, _P, _P]
            lib.fmm_tree_export_systems.restype = C.c_int
            lib.fmm_tree_set_positions.argtypes = [_P, _P, C.c_int, _P]
            lib.fmm_tree_set_positions.restype = C.c_int
            lib.fmm_backward.argtypes = [_P, _P, _P, _P, _P, _P, C.c_int, _P]
            lib.fmm_backward.restype = C.c_int
            lib.fmm_inject_dependency.argtypes = [_P, C.c_int32, C.c_int32, C.c_int32]
            lib.fmm_inject_dependency.restype = C.c_int
            lib.fmm_direct_noalloc.argtypes = [C.c_int64, _P, _P, _P, _P, C.c_int, C.c_int32, _P]
            lib.fmm_direct_noalloc.restype = C.c_int
            lib.fmm_direct_noalloc_max_n.argtypes = []
            lib.fmm_direct_noalloc_max_n.restype = C.c_int64
            for name in ("fmm_build_tree", "fmm_evaluate", "fmm_build_tree_batched", "fmm_evaluate_batched",
                         "fmm_tree_get_info", "fmm_tree_export", "fmm_status"):
                getattr(lib, name).restype = C.c_int
            _lib = lib
    return _lib


def _check(rc: int):
    if rc != FMM_OK:
        raise FMMError(rc, load().fmm_last_error().decode())


def _torch():
    import torch
    return torch


def _stream_ptr(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _dtype_code(t) -> int:
    torch = _torch()
    if t.dtype == torch.float64:
        return F64
    if t.dtype == torch.float32:
        return F32
    raise TypeError(f"unsupported dtype {t.dtype} (float64 or float32)")


class Tree:
    """A built octree with interaction lists, owned by the library."""

    def __init__(self, pos, p: int = 4, leaf_size: int = 64, theta: float = 0.5,
                 precision: int = PREC_FP64, flags: int = 0, timeout_ns: int = 0, stream=None, offsets=None,
                 p2p_item_records: int = 0, tc_min_pairs: int = 0):
        torch = _torch()
        lib = load()
        if not (pos.is_cuda and pos.dim() == 2 and pos.shape[1] == 3):
            raise ValueError("pos must be a CUDA tensor of shape (n, 3)")
        self._pos_key = _tensor_key(pos)
        pos = pos.contiguous()
        self.params = Params(int(p), int(leaf_size), float(theta), int(precision), int(flags), int(timeout_ns),
                             int(p2p_item_records), int(tc_min_pairs))
        self.n = int(pos.shape[0])
        self.device = pos.device
        h = _P()
        with torch.cuda.device(pos.device):
            if offsets is None:
                _check(lib.fmm_build_tree(C.byref(self.params), self.n, C.c_void_p(pos.data_ptr()),
                                          _dtype_code(pos), C.byref(h), _stream_ptr(stream)))
                self.offsets = np.array([0, self.n], dtype=np.int64)
            else:
                off = np.ascontiguousarray(offsets, dtype=np.int64)
                if off.ndim != 1 or off[-1] != self.n:
                    raise ValueError("offsets must be 1-D and end at n")
                _check(lib.fmm_build_tree_batched(C.byref(self.params), len(off) - 1, off.ctypes.data_as(_P),
                                                  C.c_void_p(pos.data_ptr()), _dtype_code(pos), C.byref(h),
                                                  _stream_ptr(stream)))
                self.offsets = off
        self._h = h

    # -- evaluation -------------------------------------------------------
    def evaluate(self, q, phi=None, force=None, want_phi: bool = True, want_force: bool = True, stream=None):
        """Potentials and forces (in the caller's particle order) for charges q."""
        torch = _torch()
        if not (q.is_cuda and q.dim() == 1 and q.shape[0] == self.n):
            raise ValueError("q must be a CUDA tensor of shape (n,)")
        q = q.contiguous()
        if want_phi and phi is None:
            phi = torch.empty(self.n, dtype=q.dtype, device=q.device)
        if want_force and force is None:
            force = torch.empty((self.n, 3), dtype=q.dtype, device=q.device)
        for t in (phi, force):
            if t is not None and (t.dtype != q.dtype or not t.is_contiguous()):
                raise ValueError("outputs must be contiguous and of the charges' dtype")
        with torch.cuda.device(q.device):
            _check(load().fmm_evaluate(self._h, C.c_void_p(q.data_ptr()),
                                       C.c_void_p(phi.data_ptr()) if phi is not None else None,
                                       C.c_void_p(force.data_ptr()) if force is not None else None,
                                       _dtype_code(q), _stream_ptr(stream)))
        return phi, force

    def status(self) -> int:
        return load().fmm_status(self._h)

    def inject_dependency(self, counter: int, cell: int, delta: int = 1):
        """Raise a task-queue dependency counter (failure-detection tests)."""
        _check(load().fmm_inject_dependency(self._h, int(counter), int(cell), int(delta)))

    def stage_times(self) -> dict:
        """Per-stage device ms of the last build and evaluation (tree built with TIMING)."""
        ms = np.zeros(len(STAGE_NAMES))
        _check(load().fmm_stage_times(self._h, ms.ctypes.data_as(_P), len(ms)))
        return {name: float(v) for name, v in zip(STAGE_NAMES, ms) if v >= 0}

    def kernel_launches(self, build: bool = False) -> int:
        return int(load().fmm_kernel_launches(self._h, 1 if build else 0))

    # -- inspection -------------------------------------------------------
    def info(self) -> TreeInfo:
        i = TreeInfo()
        _check(load().fmm_tree_get_info(self._h, C.byref(i)))
        return i

    def export_systems(self):
        """(origins [nsys,3], sides [nsys], cell_system [ncell]) of a batched tree."""
        i = self.info()
        ns = int(i.nsys)
        org, sd, cs = np.zeros((ns, 3)), np.zeros(ns), np.zeros(i.ncell, np.int32)
        _check(load().fmm_tree_export_systems(self._h, org.ctypes.data_as(_P), sd.ctypes.data_as(_P),
                                              cs.ctypes.data_as(_P)))
        return org, sd, cs

    def export(self) -> dict:
        """Host copies of keys, permutation, cell table and the sorted lists."""
        i = self.info()
        n, nc = i.n, i.ncell
        out = {
            "keys": np.zeros(n, np.uint64), "perm": np.zeros(n, np.int64),
            "level": np.zeros(nc, np.int32), "cell_key": np.zeros(nc, np.uint64),
            "first": np.zeros(nc, np.int64), "count": np.zeros(nc, np.int64),
            "parent": np.zeros(nc, np.int32), "child_first": np.zeros(nc, np.int32),
            "child_count": np.zeros(nc, np.int32),
            "m2l": np.zeros((i.nm2l, 2), np.int32), "p2p": np.zeros((i.np2p, 2), np.int32),
        }
        order = ["keys", "perm", "level", "cell_key", "first", "count", "parent", "child_first",
                 "child_count", "m2l", "p2p"]
        _check(load().fmm_tree_export(self._h, *[out[k].ctypes.data_as(_P) for k in order]))
        out["origin"] = np.array(i.origin[:])
        out["side"] = i.side
        return out

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            load().fmm_tree_destroy(h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def build_tree(pos, **params) -> Tree:
    return Tree(pos, **params)


def build_tree_batched(pos, offsets, **params) -> Tree:
    """One tree holding independent systems; pos holds them back to back, system s
    being rows offsets[s]..offsets[s+1]-1.  Evaluate it like any tree."""
    return Tree(pos, offsets=offsets, **params)


def capture_graph(tree, q, phi, force):
    """Capture tree.evaluate(q) into a CUDA graph writing phi and force; returns
    the torch.cuda.CUDAGraph (replay() re-runs the evaluation, which allocates
    nothing and never synchronises)."""
    torch = _torch()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        tree.evaluate(q, phi=phi, force=force)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        tree.evaluate(q, phi=phi, force=force)
    return g


def autotune_leaf_size(pos, q, offsets=None, candidates=(24, 32, 48, 64, 96, 128), repeats: int = 3, **params):
    """Time build + evaluate for each leaf size and return (best, {leaf: ms}).

    The cost balance between P2P (grows with the leaf size) and M2L (grows
    with the number of cells) depends on the distribution and the order, so
    the leaf size is chosen by measurement on the actual input."""
    torch = _torch()
    times = {}
    for leaf in candidates:
        kw = dict(params, leaf_size=int(leaf))
        best = float("inf")
        for r in range(repeats + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            t = Tree(pos, offsets=offsets, **kw)
            t.evaluate(q)
            e1.record()
            torch.cuda.synchronize()
            t.close()
            if r > 0:
                best = min(best, e0.elapsed_time(e1))
        times[int(leaf)] = best
    return min(times, key=times.get), times


def _time_build_evaluate(pos, q, offsets, repeats, kw):
    """Best of `repeats` timed build + evaluate runs (after one untimed run), ms."""
    torch = _torch()
    best = float("inf")
    for r in range(repeats + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        t = Tree(pos, offsets=offsets, **kw)
        t.evaluate(q)
        e1.record()
        torch.cuda.synchronize()
        t.close()
        if r > 0:
            best = min(best, e0.elapsed_time(e1))
    return best


def autotune(pos, q, offsets=None, leaf_sizes=(32, 48, 64, 96), p2p_item_records=(16, 32, 64, 128, 256),
             tc_min_pairs=(16, 32, 64, 128, 256), repeats: int = 2, **params):
    """Choose the work shape by measurement on the actual input: the leaf size
    (the P2P / M2L balance), the records per P2P work item of a split leaf (the
    near-field load balance) and, for the mixed form, the smallest translation
    class worth a tensor-core operator.  One coordinate sweep in that order,
    each starting from the best values found so far.  Returns (best keyword
    arguments for build_tree, {(name, value): ms}).  Every candidate computes
    the same pair interactions; only the schedule differs."""
    best = dict(params)
    best.setdefault("leaf_size", 64)
    times = {}
    sweeps = [("leaf_size", leaf_sizes), ("p2p_item_records", p2p_item_records)]
    if params.get("precision", PREC_FP64) == PREC_MIXED_TC:
        sweeps.append(("tc_min_pairs", tc_min_pairs))
    for name, values in sweeps:
        scored = {}
        for v in values:
            kw = dict(best, **{name: int(v)})
            scored[int(v)] = times[(name, int(v))] = _time_build_evaluate(pos, q, offsets, repeats, kw)
        best[name] = min(scored, key=scored.get)
    return best, times


def evaluate(tree: Tree, q, **kw):
    return tree.evaluate(q, **kw)


def version() -> str:
    return load().fmm_version().decode()


def _tensor_key(t):
    """Identity of a tensor's contents: storage address, shape and in-place version."""
    return (t.data_ptr(), tuple(t.shape), t.dtype, t._version)


def _set_positions(self, pos, stream=None):
    """Move the particles without rebuilding the tree (cells and lists stay)."""
    torch = _torch()
    if not (pos.is_cuda and pos.shape == (self.n, 3)):
        raise ValueError("pos must be a CUDA tensor of shape (n, 3)")
    self._pos_key = _tensor_key(pos)
    pos = pos.contiguous()
    with torch.cuda.device(pos.device):
        _check(load().fmm_tree_set_positions(self._h, C.c_void_p(pos.data_ptr()), _dtype_code(pos),
                                             _stream_ptr(stream)))


def _backward(self, q, w, field_q, stream=None):
    """(dL/dq, dL/dx) of L = sum w_i phi_i, from one adjoint FMM pass (tree built with OUT_FIELD)."""
    torch = _torch()
    q, w, field_q = q.contiguous(), w.contiguous(), field_q.contiguous()
    dq = torch.empty_like(q)
    dx = torch.empty((self.n, 3), dtype=q.dtype, device=q.device)
    with torch.cuda.device(q.device):
        _check(load().fmm_backward(self._h, C.c_void_p(q.data_ptr()), C.c_void_p(w.data_ptr()),
                                   C.c_void_p(field_q.data_ptr()), C.c_void_p(dq.data_ptr()),
                                   C.c_void_p(dx.data_ptr()), _dtype_code(q), _stream_ptr(stream)))
    return dq, dx


Tree.set_positions = _set_positions
Tree.backward = _backward


def _fmm_function():
    import torch

    class FMMFunction(torch.autograd.Function):
        """phi = FMM(pos, q) as an autograd node.

        ``tree`` must be built on ``pos`` with OUT_FIELD (the forward keeps the
        field for the backward).  The backward runs one more FMM pass with the
        upstream gradient as charges (the kernel is symmetric) and returns
        dL/dpos and dL/dq; the tree is held fixed, so positions are treated as
        moving inside their cells.  ``pos`` must have the tree's shape; when it
        is not the tensor the tree was built on (another tensor, or the same one
        changed in place since), the tree takes its values first
        (``Tree.set_positions``: same cells and lists, particles moved), so phi
        and the gradients are always those of ``pos``."""

        @staticmethod
        def forward(ctx, pos, q, tree):
            if not (tree.params.flags & OUT_FIELD):
                raise ValueError("FMMFunction needs a tree built with flags=OUT_FIELD")
            if tuple(pos.shape) != (tree.n, 3) or tuple(q.shape) != (tree.n,):
                raise ValueError(f"pos must be ({tree.n}, 3) and q ({tree.n},) for this tree")
            if _tensor_key(pos) != tree._pos_key:
                tree.set_positions(pos.detach())
            phi, field = tree.evaluate(q)
            ctx.tree = tree
            ctx.save_for_backward(q, field)
            return phi

        @staticmethod
        def backward(ctx, w):
            q, field = ctx.saved_tensors
            dq, dx = ctx.tree.backward(q, w.contiguous().to(q.dtype), field)
            return dx, dq, None

    return FMMFunction


def __getattr__(name):
    if name == "FMMFunction":
        return _fmm_function()
    raise AttributeError(name)
