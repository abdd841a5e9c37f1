"""Work-shape tunables (fmm_params.p2p_item_records, tc_min_pairs) and the
autotuner: every shape computes the same pair interactions, so values agree
up to summation order, and the autotuner returns a candidate of each sweep."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.gpu_common import gpu_eval, gpu_tree, torch_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("records", [8, 16, 1024])
def test_p2p_item_records_fp64_same_values(records):
    """FP64 stage by stage: splitting the near-field lists into runs of any
    length changes only the FP64 summation order of the split leaves."""
    import paper_1203_0889_gb300 as fmm
    wl = W.make_workload("clustered", n=30000)
    ref = gpu_tree(wl.pos, p=6, leaf_size=32, theta=0.5, precision=fmm.PREC_FP64, flags=fmm.STAGED)
    t = gpu_tree(wl.pos, p=6, leaf_size=32, theta=0.5, precision=fmm.PREC_FP64, flags=fmm.STAGED,
                 p2p_item_records=records)
    assert np.array_equal(ref.export()["p2p"], t.export()["p2p"])
    p0, f0 = gpu_eval(ref, wl.q)
    p1, f1 = gpu_eval(t, wl.q)
    assert O.rel_l2(p1, p0) <= 1e-13 and O.rel_l2(f1, f0) <= 1e-13


@pytest.mark.parametrize("records,min_pairs", [(8, 1), (32, 16), (1024, 256), (64, 4096)])
def test_mixed_shapes_same_values(records, min_pairs):
    """Mixed form: the classes left to the CUDA cores and the P2P split change
    the FP32 summation order only (and the tensor cores' share of the pairs)."""
    import paper_1203_0889_gb300 as fmm
    wl = W.make_workload("clustered", n=50000)
    ref = gpu_tree(wl.pos, p=10, leaf_size=64, theta=0.5, precision=fmm.PREC_MIXED_TC)
    t = gpu_tree(wl.pos, p=10, leaf_size=64, theta=0.5, precision=fmm.PREC_MIXED_TC, p2p_item_records=records,
                 tc_min_pairs=min_pairs)
    assert np.array_equal(ref.export()["m2l"], t.export()["m2l"])
    a, b = ref.info(), t.info()
    assert b.tc_pairs <= a.tc_pairs if min_pairs >= 64 else b.tc_pairs >= a.tc_pairs
    p0, f0 = gpu_eval(ref, wl.q)
    p1, f1 = gpu_eval(t, wl.q)
    assert t.status() == fmm.FMM_OK
    assert O.rel_l2(p1, p0) <= 2e-6 and O.rel_l2(f1, f0) <= 2e-6, (O.rel_l2(p1, p0), O.rel_l2(f1, f0))


def test_autotune_returns_candidates():
    import paper_1203_0889_gb300 as fmm
    torch, dev = torch_dev()
    wl = W.make_workload("clustered", n=40000)
    pos = torch.tensor(wl.pos, dtype=torch.float64, device=dev)
    q = torch.tensor(wl.q, dtype=torch.float64, device=dev)
    best, times = fmm.autotune(pos, q, leaf_sizes=(32, 64), p2p_item_records=(16, 64), tc_min_pairs=(32, 64),
                               repeats=1, p=8, theta=0.5, precision=fmm.PREC_MIXED_TC)
    assert best["leaf_size"] in (32, 64) and best["p2p_item_records"] in (16, 64)
    assert best["tc_min_pairs"] in (32, 64)
    assert len(times) == 6 and all(v > 0 for v in times.values())
    t = fmm.build_tree(pos, **best)
    phi, f = t.evaluate(q)
    torch.cuda.synchronize()
    assert t.status() == fmm.FMM_OK and bool(torch.isfinite(phi).all())


def test_granularity_study_small():
    """The task-granularity study (task queue, N against leaf size) runs on the
    GPU and reports a row per configuration with a clean status."""
    import json
    import subprocess
    import sys
    r = subprocess.run([sys.executable, "bench.py", "--workload", "granularity", "--granularity-n", "20000,60000",
                        "--granularity-p", "6", "--granularity-leaf", "16,64"], capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    rows = out["rows"]
    assert len(rows) == 4
    for row in rows:
        assert row["status"] == 0 and row["particles_per_s"] > 0 and row["tasks"] > 0
    # more, smaller tasks at the smaller leaf size
    by = {(row["n"], row["leaf"]): row for row in rows}
    assert by[(60000, 16)]["tasks"] > by[(60000, 64)]["tasks"]
