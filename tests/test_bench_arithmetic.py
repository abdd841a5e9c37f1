"""bench.py's roofline arithmetic on the CPU: the algorithmic units behind
`achieved` and `frac` (pair counts, flops, bytes) against brute force and hand
arithmetic on small oracle trees."""
import itertools
import types

import numpy as np

import bench
import oracle as O
import workloads as W


def _export(ref):
    """The fields of a tree export that the bench helpers read."""
    return {"count": ref.count.astype(np.int64), "p2p": ref.p2p, "m2l": ref.m2l, "keys": ref.keys,
            "child_count": ref.child_count.astype(np.int64)}


def test_p2p_pairs_is_the_number_of_near_field_particle_pairs():
    """sum over P2P leaf pairs of |A||B| minus the N self pairs = the ordered
    particle pairs (i != j) whose leaves form a P2P pair, counted one by one."""
    pos = W.make_workload("plummer", n=700).pos
    ref = O.build_tree(pos, 16, 0.5)
    leaf_of = np.empty(ref.n, dtype=np.int64)
    for c in np.nonzero(ref.child_count == 0)[0]:
        leaf_of[ref.first[c]:ref.first[c] + ref.count[c]] = c
    near = {(int(a), int(b)) for a, b in ref.p2p}
    brute = sum(1 for i, j in itertools.permutations(range(ref.n), 2) if (leaf_of[i], leaf_of[j]) in near)
    assert bench.p2p_pairs(_export(ref)) == brute


def test_kernel_rooflines_arithmetic():
    ref = O.build_tree(W.make_workload("uniform", n=3000).pos, 32, 0.5)
    ex = _export(ref)
    pairs = bench.p2p_pairs(ex)
    K = (bench.P + 1) ** 2
    ki = (K + 63) // 64 * 64
    info = types.SimpleNamespace(tc_pairs=len(ref.m2l), tc_items=(len(ref.m2l) + 127) // 128)
    stage_ms = {"p2p": 2.0, "m2l_tc": 4.0, "m2l": 4.5}
    roofs = {r["kernel"]: r for r in bench.kernel_rooflines(stage_ms, ex, 3, 152, info)}
    p2p = roofs["k_p2p"]
    assert np.isclose(p2p["achieved"], pairs * bench.P2P_FLOPS_PER_PAIR / 2e-3 / 1e12)
    assert np.isclose(p2p["peak"], 152 * 128 * 2 * 2070e6 / 1e12, rtol=0.05)
    assert np.isclose(p2p["frac"], p2p["achieved"] / p2p["peak"])
    tc = roofs["k_m2l_tc"]
    assert np.isclose(tc["achieved"], len(ref.m2l) * 2.0 * K * K / 4e-3 / 1e12)
    assert np.isclose(tc["frac"], tc["achieved"] / tc["peak"])
    assert np.isclose(tc["issued_frac"] * tc["peak"], info.tc_items * 3 * 2.0 * 128 * 128 * ki / 4e-3 / 1e12)
    # FP64 and FP32 task-queue forms: one entry, M2L and P2P flops over the queue time
    q = bench.kernel_rooflines({"queue": 10.0}, ex, 0, 152)
    assert len(q) == 1 and q[0]["kernel"] == "k_queue"
    flops = len(ref.m2l) * 2.0 * K * K + pairs * bench.P2P_FLOPS_PER_PAIR
    assert np.isclose(q[0]["achieved"], flops / 10e-3 / 1e12)
    assert q[0]["peak"] == bench.FP64_TFLOPS_MEASURED


def test_pass_rooflines_bytes():
    ref = O.build_tree(W.make_workload("clustered", n=2000).pos, 16, 0.5)
    ex = _export(ref)
    n = ref.n
    K = (bench.P + 1) ** 2
    stage_ms = {"p2m": 0.1, "m2m": 0.2, "l2l": 0.3, "l2p": 0.4}
    got = {r["stage"]: r for r in bench.pass_rooflines(stage_ms, ex, 3, None, n)}
    cc = ref.child_count
    nleaf = int((cc == 0).sum())
    b = 4   # FP32 expansions in the mixed form
    assert got["p2m"]["bytes"] == 16 * n + nleaf * K * b
    assert got["m2m"]["bytes"] == sum((int(c) + 1) * K * b for c in cc if c > 0)
    assert got["l2l"]["bytes"] == 3 * K * b * (len(cc) - 1)
    assert got["l2p"]["bytes"] == 32 * n + nleaf * K * b
    for name, r in got.items():
        assert np.isclose(r["achieved"], r["bytes"] / (stage_ms[name] * 1e-3) / 1e9)
        assert np.isclose(r["frac"], r["achieved"] / r["peak"])
