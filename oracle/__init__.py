"""CPU FP64 oracle for the adaptive 3-D Laplace FMM -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its binding) never does.  The arithmetic lives in ``fmm_oracle.c`` (plain C,
FP64, compiled without FMA contraction); this module compiles it with gcc and
marshals arrays through ctypes.

Functions and what they follow:

* ``direct`` / ``direct_targets`` -- the exact sum the FMM approximates
  (Section 2.1: the N-body interaction; potential q_j / r, field gradient).
* ``build_tree`` -- root cube, 21-bit quantisation, Morton keys (Section 2.2),
  adaptive octree with bounded leaf population (Section 2.1), breadth-first
  dual tree traversal with the size/distance acceptance test (Sections 4, 5).
* ``fmm_evaluate`` -- P2M, M2M, M2L, L2L, L2P, P2P in the order of the stage
  flow of Section 2.1.
* ``p2m``, ``m2m``, ``m2l``, ``l2l``, ``l2p``, ``m2p`` -- single operators,
  used by the pins (complex coefficients, index n*n + n + m, m = -n..n).
* ``uvwx`` (submodule) -- the parent-neighbour-child lists U, V, W, X of
  Section 2.1's alternative separation rule and the potential through them.
* ``force_grad`` (submodule) -- the direct-sum gradient of a loss on
  potentials and forces (what a backward for force-dependent losses computes).
"""
from __future__ import annotations

import contextlib
import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fmm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, no fast-math)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-o", tmp, _SRC, "-lm", "-lpthread"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Tree(C.Structure):
    _fields_ = [
        ("n", C.c_int64), ("p_unused", C.c_int32), ("ncell", C.c_int32),
        ("nm2l", C.c_int64), ("np2p", C.c_int64), ("nlevel", C.c_int32),
        ("leaf_size", C.c_int32), ("theta", C.c_double), ("origin", C.c_double * 3),
        ("side", C.c_double),
        ("keys", C.POINTER(C.c_uint64)), ("perm", C.POINTER(C.c_int64)),
        ("level", C.POINTER(C.c_int32)), ("cell_key", C.POINTER(C.c_uint64)),
        ("first", C.POINTER(C.c_int64)), ("count", C.POINTER(C.c_int64)),
        ("parent", C.POINTER(C.c_int32)), ("child_first", C.POINTER(C.c_int32)),
        ("child_count", C.POINTER(C.c_int32)),
        ("m2l", C.POINTER(C.c_int32)), ("p2p", C.POINTER(C.c_int32)),
    ]


_P = C.c_void_p


def _configure(lib):
    lib.oracle_build_tree.restype = C.POINTER(_Tree)
    lib.oracle_build_tree.argtypes = [C.c_int64, _P, C.c_int32, C.c_double]
    lib.oracle_free_tree.argtypes = [C.POINTER(_Tree)]
    lib.oracle_fmm_evaluate.argtypes = [C.POINTER(_Tree), _P, C.c_int, _P, _P, _P, C.c_int]
    lib.oracle_fmm_evaluate_leaves.argtypes = [C.POINTER(_Tree), _P, C.c_int, _P, C.c_int64, _P, _P, _P]
    lib.oracle_direct.argtypes = [C.c_int64, _P, _P, _P, _P]
    lib.oracle_direct_targets.argtypes = [C.c_int64, _P, _P, C.c_int64, _P, _P, _P]
    lib.oracle_p2m.argtypes = [C.c_int, _P, C.c_int64, _P, _P, _P]
    lib.oracle_m2m.argtypes = [C.c_int, _P, _P, _P]
    lib.oracle_m2l.argtypes = [C.c_int, _P, _P, _P]
    lib.oracle_l2l.argtypes = [C.c_int, _P, _P, _P]
    lib.oracle_l2p.argtypes = [C.c_int, _P, _P, _P, _P]
    lib.oracle_m2p.argtypes = [C.c_int, _P, _P, _P]
    return lib


def compile_variant(source_text: str, out_path: str) -> str:
    """Compile a modified copy of the oracle source (used by the tests that
    plant mistakes in the oracle to show that the pins catch them)."""
    src = out_path + ".c"
    with open(src, "w") as f:
        f.write(source_text)
    subprocess.run(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
                    "-fno-fast-math", "-o", out_path, src, "-lm", "-lpthread"], check=True)
    return out_path


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


@contextlib.contextmanager
def using_library(path: str):
    """Temporarily route every call of this module to another build of the oracle."""
    global _lib
    with _lock:
        old = _lib
        _lib = _configure(C.CDLL(path))
    try:
        yield
    finally:
        with _lock:
            _lib = old


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            _configure(lib)
            _lib = lib
    return _lib


def _d(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


class Tree:
    """Host copy of the oracle's tree: keys, permutation, cell table, lists."""

    def __init__(self, pos, leaf_size: int, theta: float):
        lib = _load()
        self.pos = _d(pos, (-1, 3))
        self.n = self.pos.shape[0]
        self._t = lib.oracle_build_tree(self.n, _ptr(self.pos), int(leaf_size), float(theta))
        t = self._t.contents
        n, nc = t.n, t.ncell

        def arr(p, cnt, dt):
            if cnt == 0:
                return np.zeros(0, dtype=dt)
            return np.ctypeslib.as_array(p, shape=(cnt,)).astype(dt, copy=True)

        self.leaf_size, self.theta = int(leaf_size), float(theta)
        self.origin = np.array(t.origin[:])
        self.side = float(t.side)
        self.ncell = nc
        self.nlevel = t.nlevel
        self.keys = arr(t.keys, n, np.uint64)
        self.perm = arr(t.perm, n, np.int64)
        self.level = arr(t.level, nc, np.int32)
        self.cell_key = arr(t.cell_key, nc, np.uint64)
        self.first = arr(t.first, nc, np.int64)
        self.count = arr(t.count, nc, np.int64)
        self.parent = arr(t.parent, nc, np.int32)
        self.child_first = arr(t.child_first, nc, np.int32)
        self.child_count = arr(t.child_count, nc, np.int32)
        self.m2l = arr(t.m2l, 2 * t.nm2l, np.int32).reshape(-1, 2)
        self.p2p = arr(t.p2p, 2 * t.np2p, np.int32).reshape(-1, 2)

    def __del__(self):
        try:
            if getattr(self, "_t", None):
                _load().oracle_free_tree(self._t)
                self._t = None
        except Exception:
            pass

    @property
    def is_leaf(self):
        return self.child_count == 0

    def centres(self) -> np.ndarray:
        """Geometric cell centres in input coordinates (same formula as the C code)."""
        kc = np.zeros((self.ncell, 3), dtype=np.int64)
        for b in range(21):
            for d in range(3):
                kc[:, d] |= ((self.cell_key >> np.uint64(3 * b + d)) & np.uint64(1)).astype(np.int64) << b
        s = (np.int64(1) << (21 - self.level.astype(np.int64)))
        twoc = 2 * kc * s[:, None] + s[:, None]
        return self.origin[None, :] + twoc.astype(np.float64) * (self.side / 4194304.0)

    def evaluate(self, p: int, q, nthreads: int = 1):
        """Full FMM; returns (phi[n], grad_phi[n,3]) in input order."""
        q = _d(q)
        phi = np.zeros(self.n)
        grad = np.zeros((self.n, 3))
        _load().oracle_fmm_evaluate(self._t, _ptr(self.pos), int(p), _ptr(q), _ptr(phi), _ptr(grad), int(nthreads))
        return phi, grad

    def evaluate_leaves(self, p: int, q, leaves):
        """FMM result for the particles of the given leaves only.

        Returns (input_indices, phi, grad) with the particles in sorted order,
        leaf after leaf."""
        q = _d(q)
        leaves = np.ascontiguousarray(leaves, dtype=np.int32)
        cnt = int(self.count[leaves].sum())
        phi = np.zeros(cnt)
        grad = np.zeros((cnt, 3))
        _load().oracle_fmm_evaluate_leaves(self._t, _ptr(self.pos), int(p), _ptr(q), len(leaves),
                                           _ptr(leaves), _ptr(phi), _ptr(grad))
        idx = np.concatenate([self.perm[self.first[c]:self.first[c] + self.count[c]] for c in leaves]) \
            if len(leaves) else np.zeros(0, np.int64)
        return idx, phi, grad


def build_tree(pos, leaf_size: int = 64, theta: float = 0.5) -> Tree:
    return Tree(pos, leaf_size, theta)


def fmm_evaluate(pos, q, p: int = 4, leaf_size: int = 64, theta: float = 0.5, nthreads: int = 1):
    t = Tree(pos, leaf_size, theta)
    return t.evaluate(p, q, nthreads)


def direct(pos, q):
    """O(N^2) FP64 direct sum: (phi, grad_phi), r = 0 pairs skipped."""
    pos, q = _d(pos, (-1, 3)), _d(q)
    n = pos.shape[0]
    phi, grad = np.zeros(n), np.zeros((n, 3))
    _load().oracle_direct(n, _ptr(pos), _ptr(q), _ptr(phi), _ptr(grad))
    return phi, grad


def direct_targets(pos, q, targets):
    pos, q = _d(pos, (-1, 3)), _d(q)
    targets = np.ascontiguousarray(targets, dtype=np.int64)
    phi, grad = np.zeros(len(targets)), np.zeros((len(targets), 3))
    _load().oracle_direct_targets(pos.shape[0], _ptr(pos), _ptr(q), len(targets), _ptr(targets),
                                  _ptr(phi), _ptr(grad))
    return phi, grad


# ---- single operators (complex coefficients, full m range) ----

def ncoef(p: int) -> int:
    return (p + 1) * (p + 1)


def hidx(n: int, m: int) -> int:
    return n * n + n + m


def p2m(p, centre, pos, q):
    pos, q, c = _d(pos, (-1, 3)), _d(q), _d(centre)
    M = np.zeros(ncoef(p), dtype=np.complex128)
    _load().oracle_p2m(int(p), _ptr(c), pos.shape[0], _ptr(pos), _ptr(q), _ptr(M))
    return M


def m2m(p, Mc, d):
    Mp = np.zeros(ncoef(p), dtype=np.complex128)
    Mc = np.ascontiguousarray(Mc, dtype=np.complex128)
    _load().oracle_m2m(int(p), _ptr(Mc), _ptr(_d(d)), _ptr(Mp))
    return Mp


def m2l(p, M, D):
    L = np.zeros(ncoef(p), dtype=np.complex128)
    M = np.ascontiguousarray(M, dtype=np.complex128)
    _load().oracle_m2l(int(p), _ptr(M), _ptr(_d(D)), _ptr(L))
    return L


def l2l(p, Lp, d):
    Lc = np.zeros(ncoef(p), dtype=np.complex128)
    Lp = np.ascontiguousarray(Lp, dtype=np.complex128)
    _load().oracle_l2l(int(p), _ptr(Lp), _ptr(_d(d)), _ptr(Lc))
    return Lc


def l2p(p, L, y):
    L = np.ascontiguousarray(L, dtype=np.complex128)
    phi = np.zeros(1)
    g = np.zeros(3)
    _load().oracle_l2p(int(p), _ptr(L), _ptr(_d(y)), _ptr(phi), _ptr(g))
    return float(phi[0]), g


def m2p(p, M, y):
    M = np.ascontiguousarray(M, dtype=np.complex128)
    phi = np.zeros(1)
    _load().oracle_m2p(int(p), _ptr(M), _ptr(_d(y)), _ptr(phi))
    return float(phi[0])


def rel_l2(a, b) -> float:
    a, b = np.asarray(a, np.float64).ravel(), np.asarray(b, np.float64).ravel()
    den = float(np.sum(b * b))
    return float(np.sqrt(np.sum((a - b) ** 2) / den)) if den > 0 else float(np.sqrt(np.sum((a - b) ** 2)))
