"""The GPU U/V/W/X list builder's functions (csrc/uvwx.cuh), compiled for the
host with nvcc, against the oracle's lists built from their definitions
(oracle/uvwx.py) on the same trees: the M2L pairs (V) and the P2P pairs (U,
and W / X as direct sums) must be the same sets, with no duplicates.  The
kernels of uvwx.cu call these functions per cell and per leaf in the same
order; this check needs no GPU."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle import uvwx

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1203_0889_gb300", "csrc")


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("uvwx") / "uvwx_host_check")
    subprocess.run([nvcc, "-std=c++17", "-O1", "-I", CSRC, os.path.join(ROOT, "tests", "uvwx_host_check.cu"),
                    "-o", exe], check=True, capture_output=True)
    return exe


def _dump(t, path):
    """The tree's arrays in the device layout: doubled integer centres, level."""
    kc = np.zeros((t.ncell, 3), dtype=np.int64)
    for b in range(21):
        for d in range(3):
            kc[:, d] |= ((t.cell_key >> np.uint64(3 * b + d)) & np.uint64(1)).astype(np.int64) << b
    s = np.int64(1) << (21 - t.level.astype(np.int64))
    ic = np.concatenate([2 * kc * s[:, None] + s[:, None], t.level[:, None].astype(np.int64)], axis=1)
    leaves = np.nonzero(t.child_count == 0)[0]
    pleaf = np.zeros(t.n, np.int64)
    for c in leaves:
        pleaf[t.first[c]:t.first[c] + t.count[c]] = c
    ls = np.searchsorted(t.level, np.arange(t.nlevel + 1), "left")
    assert np.all(np.diff(t.level) >= 0)
    i32 = lambda a: np.asarray(a, dtype=np.int32).tobytes()   # noqa: E731
    with open(path, "wb") as f:
        f.write(i32([t.ncell, len(leaves), t.n, t.nlevel]))
        f.write(i32(ls))
        f.write(i32(ic))
        for a in (t.parent, t.child_first, t.child_count, t.first, t.count, leaves, pleaf):
            f.write(i32(a))


def _run(harness, t, tmp_path):
    src, out = str(tmp_path / "tree.bin"), str(tmp_path / "pairs.bin")
    _dump(t, src)
    r = subprocess.run([harness, src, out], capture_output=True)
    assert r.returncode == 0, r
    raw = open(out, "rb").read()
    nm, np_ = np.frombuffer(raw[:16], dtype=np.int64)
    pairs = np.frombuffer(raw[16:], dtype=np.int32).reshape(-1, 2)
    return pairs[:nm], pairs[nm:nm + np_]


@pytest.mark.parametrize("name,n,leaf", [("uniform", 1500, 16), ("plummer", 1500, 8), ("clustered", 2000, 16),
                                         ("clustered", 800, 1)])
def test_host_build_matches_oracle_lists(harness, tmp_path, name, n, leaf):
    wl = W.make_workload(name, n=n)
    t = O.build_tree(wl.pos, leaf, 0.5)
    m2l, p2p = _run(harness, t, tmp_path)
    ref_m2l, ref_p2p = uvwx.pair_lists(t)
    assert len(set(map(tuple, p2p.tolist()))) == len(p2p)        # no pair twice
    assert len(set(map(tuple, m2l.tolist()))) == len(m2l)
    assert np.array_equal(np.array(sorted(map(tuple, m2l.tolist())), dtype=np.int32).reshape(-1, 2), ref_m2l)
    assert np.array_equal(np.array(sorted(map(tuple, p2p.tolist())), dtype=np.int32).reshape(-1, 2), ref_p2p)


def test_host_build_deep_branch(harness, tmp_path):
    """A dense corner beside sparse particles: a deep branch next to coarse
    leaves (long descents, many W cells)."""
    rng = np.random.default_rng(9)
    pos = np.concatenate([1e-4 * rng.random((400, 3)), [[1.0, 1.0, 1.0]], rng.random((200, 3))])
    t = O.build_tree(pos, 8, 0.5)
    m2l, p2p = _run(harness, t, tmp_path)
    ref_m2l, ref_p2p = uvwx.pair_lists(t)
    assert np.array_equal(np.array(sorted(map(tuple, p2p.tolist())), dtype=np.int32).reshape(-1, 2), ref_p2p)
    assert np.array_equal(np.array(sorted(map(tuple, m2l.tolist())), dtype=np.int32).reshape(-1, 2), ref_m2l)
