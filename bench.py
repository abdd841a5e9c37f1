#!/usr/bin/env python3
"""Benchmark: adaptive 3-D Laplace FMM on one GB300 (or N replicas).

A step is one pass of the whole hot path on one synthetic system: the device
tree build (root cube, Morton keys, octree, dual traversal, lists) followed by
one evaluation (P2M, M2M, M2L, L2L, L2P, P2P).  The default workload is the
mixed-precision configuration: N = 4,194,304 particles in 64 isotropic Gaussian
clusters (sigma = 0.01, centres uniform in the unit cube), charges U[-1, 1],
order p = 10, leaf size 64, theta = 0.5.  `--workload plummer` runs the
irregular configuration instead (N = 1,048,576 from a Plummer sphere of scale
radius 1 truncated at r = 50, charges 1/N, p = 8, leaf 64, theta = 0.4).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

The headline is the mixed form (tensor-core M2L from split bf16 products,
FP32 elsewhere, the near field in the mutual form: each pair of two different
leaves evaluated once for both), whose error against the plain FP64 GPU path
is measured in the same run and printed beside it; the FP64,
FP32-P2P/FP64-expansion and FP32 forms, the non-mutual near field and the task
graph are timed on the same system as context ("variants"), and the mixed form
of the Plummer configuration with its own error.

Prints one JSON line (rank 0).  Under torchrun each rank runs its own system
(replicas: the single-system path has no exchange step) and the value is the
particles of all ranks over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "FMM particles/sec at rel-L2 err <=1e-4 vs plain FP64 GPU path; % roofline"
# single-system workloads: description, default N, p, leaf size, theta
SYSTEMS = {
    "clustered": ("clustered: 64 Gaussian clusters sigma=0.01, centres U[0,1)^3, q~U[-1,1]", 1 << 22, 10, 64, 0.5),
    "plummer": ("plummer a=1 rmax=50, q=1/N", 1 << 20, 8, 64, 0.4),
}
WORKLOAD = "clustered"
DESC, N_DEFAULT, P, LEAF, THETA = SYSTEMS[WORKLOAD]


def select_workload(name: str) -> None:
    """Make `name` the single-system workload of this run (sets the module's
    WORKLOAD, DESC, N_DEFAULT, P, LEAF, THETA)."""
    global WORKLOAD, DESC, N_DEFAULT, P, LEAF, THETA
    WORKLOAD = name
    DESC, N_DEFAULT, P, LEAF, THETA = SYSTEMS[name]


def workload_line(n: int) -> str:
    return f"{DESC}, N={n}, p={P}, leaf={LEAF}, theta={THETA}"


def workload_seed(rank: int = 0) -> int:
    import workloads as W
    return 12030889 * 10 + W.WORKLOADS[WORKLOAD][0] + 1000 * rank
L2_FLUSH_BYTES = 512 << 20          # larger than the 129 MB L2
P2P_FLOPS_PER_PAIR = 20             # convention for the near-field direct sum
PREC_NAMES = {0: "fp64", 1: "fp32_p2p", 2: "fp32", 3: "mixed_tc"}
PREC_DTYPE = {0: "f64", 1: "f32 P2P / f64 expansions", 2: "f32", 3: "bf16x3 M2L / f32"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=None, help="particles (default: the workload's N)")
    ap.add_argument("--precision", type=int, default=3,
                    help="0 fp64, 1 fp32 P2P + fp64 expansions, 2 fp32, 3 mixed: bf16x3 tensor-core M2L + fp32")
    ap.add_argument("--no-variants", action="store_true", help="skip the other precisions' context timings")
    ap.add_argument("--staged", action="store_true", help="one kernel per stage instead of the task queue")
    ap.add_argument("--task-graph", action="store_true",
                    help="mixed form: run the evaluation as one persistent task-graph launch (FMM_TASK_GRAPH)")
    ap.add_argument("--mutual", action=argparse.BooleanOptionalAction, default=True,
                    help="mutual near field (FMM_MUTUAL): cross-leaf pairs evaluated once for both leaves "
                         "(FP32 near field, stage-by-stage evaluation; not with --task-graph)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--granularity-n", default="100000,1000000,10000000",
                    help="granularity study: particle counts (comma-separated)")
    ap.add_argument("--granularity-p", default="6,9", help="granularity study: expansion orders")
    ap.add_argument("--granularity-leaf", default="16,32,64,128,256", help="granularity study: leaf sizes")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-n", type=int, default=1 << 21,
                    help="particles of the oracle's timed sample (about 10-20 s on 16 host cores)")
    ap.add_argument("--workload", default="clustered",
                    choices=["clustered", "plummer", "batched", "table", "granularity"],
                    help="clustered: one 4M-particle clustered system at p=10 (default); plummer: one 1M-particle "
                         "Plummer system at p=8; batched: 512 systems of 1024..65536; "
                         "table: every configuration against the oracle (context, several minutes); "
                         "granularity: task size against N on the task queue")
    return ap.parse_args()


def max_over_ranks(x: float, device=None) -> float:
    """The slowest rank's value (max over the process group; x itself without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(n_per_rank: int, world: int, steps: int, slowest_s: float) -> float:
    """Particles of all ranks over the slowest rank's time (replicas: weak scaling)."""
    return n_per_rank * world * steps / slowest_s


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); smax.append(float(f[2])); power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power)}


# ---------------------------------------------------------------- our arm

def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


def p2p_pairs(ex) -> int:
    """Algorithmic near-field pair count: sum over P2P pairs |A||B| minus the N self pairs."""
    cnt = ex["count"]
    pl = ex["p2p"]
    if len(pl) == 0:
        return 0
    return int((cnt[pl[:, 0]] * cnt[pl[:, 1]]).sum() - len(ex["keys"]))


# FP64 FMA throughput of one GB300 (TFLOP/s) from a dependent-chain FMA probe
# over all SMs at the loaded clock: the FP64 pipe is narrow on this part.
FP64_TFLOPS_MEASURED = 1.256

# DRAM bytes (read + write) per launch from one ncu capture of the kernel as it
# stands; None once the kernel has changed since.
# dram__bytes_read.sum + dram__bytes_write.sum of one full-size launch of the
# kernel as it stands (one-pass ncu captures, profiles/traffic_full_size.md)
TRAFFIC = {"plummer": {"k_p2p": 89945856 + 15920640, "k_m2l_tc": 159664384 + 7156736},
           "clustered": {"k_p2p": 296624384 + 112857344, "k_m2l_tc": 14935927000 + 7914889000}}


def traffic(kernel: str):
    return TRAFFIC.get(WORKLOAD, {}).get(kernel)


def kernel_rooflines(stage_ms: dict, ex, prec: int, n_sm: int, info=None, mutual: bool = False):
    """Roofline objects of the evaluation's heavy kernels.  Their times are the
    library's own CUDA events around each stage inside the timed region,
    recorded on the stream the stage is launched on (P2P runs on the tree's
    second stream)."""
    pk, how = peaks()
    clk = float(pk.get("sm_max_mhz", 2070.0))
    fp32_peak = n_sm * 128 * 2 * clk * 1e6 / 1e12          # TFLOP/s, FP32 FMA lanes at the maximum clock
    fp32_src = f"{n_sm} SM x 128 FP32 lanes x 2 flop x {clk:.0f} MHz (derived, not measured)"
    fp64_src = "FP64 FMA probe, measured"
    K = (P + 1) ** 2
    out = []
    pairs = p2p_pairs(ex)
    if "queue" in stage_ms:
        tq = stage_ms["queue"] * 1e-3
        nm2l = len(ex["m2l"])
        flops = nm2l * 2.0 * K * K + pairs * float(P2P_FLOPS_PER_PAIR)
        peak = FP64_TFLOPS_MEASURED if prec in (0, 1) else fp32_peak
        out.append({"kernel": "k_queue", "bound": "alu", "achieved": flops / tq / 1e12, "peak": peak,
                    "unit": "TFLOP/s", "frac": flops / tq / 1e12 / peak, "traffic": None, "ms": stage_ms["queue"],
                    "algorithmic": f"{nm2l} M2L pairs x 2K^2 + {pairs} P2P pairs x {P2P_FLOPS_PER_PAIR} flops",
                    "peak_source": fp64_src if prec in (0, 1) else fp32_src})
        return out
    if "p2p" in stage_ms and pairs > 0:
        t = stage_ms["p2p"] * 1e-3
        flops = pairs * float(P2P_FLOPS_PER_PAIR)
        peak = FP64_TFLOPS_MEASURED if prec == 0 else fp32_peak
        # the mutual form does the same directed pairs' work (each cross-leaf pair once)
        kname = "k_p2p_mutual" if mutual and prec != 0 else "k_p2p"
        out.append({"kernel": kname, "bound": "alu", "achieved": flops / t / 1e12, "peak": peak,
                    "unit": "TFLOP/s", "frac": flops / t / 1e12 / peak,
                    "traffic": traffic("k_p2p") if kname == "k_p2p" else None,
                    "ms": stage_ms["p2p"],
                    "algorithmic": f"{pairs} pair interactions x {P2P_FLOPS_PER_PAIR} flops",
                    "peak_source": fp64_src if prec == 0 else fp32_src})
    if prec == 3 and info is not None and info.tc_pairs > 0 and "m2l_tc" in stage_ms:
        t = stage_ms["m2l_tc"] * 1e-3
        # issued: per 128-pair item, three bf16 products of the 128-row operator
        # (outputs padded to 128) by 128 columns (pairs) over KI inputs, KI = K
        # rounded up to whole 64-coefficient swizzle atoms
        ki = (K + 63) // 64 * 64
        useful = info.tc_pairs * 2.0 * K * K
        issued = info.tc_items * 3 * 2.0 * 128 * 128 * ki
        peak = float(pk["bf16_tflops"])
        out.append({"kernel": "k_m2l_tc", "bound": "tensor", "achieved": useful / t / 1e12, "peak": peak,
                    "unit": "TFLOP/s", "frac": useful / t / 1e12 / peak, "traffic": traffic("k_m2l_tc"),
                    "ms": stage_ms["m2l_tc"],
                    "algorithmic": f"{info.tc_pairs} M2L pairs x 2K^2 flops, K=(p+1)^2={K}",
                    "issued_frac": issued / t / 1e12 / peak,
                    "peak_source": f"bf16 dense, {how} (MEASURED_PEAKS.json burst)"})
    elif "m2l" in stage_ms:
        t = stage_ms["m2l"] * 1e-3
        nm2l = len(ex["m2l"])
        flops = nm2l * 2.0 * K * K
        peak = FP64_TFLOPS_MEASURED if prec in (0, 1) else fp32_peak
        out.append({"kernel": "k_m2l_generic", "bound": "alu", "achieved": flops / t / 1e12, "peak": peak,
                    "unit": "TFLOP/s", "frac": flops / t / 1e12 / peak, "traffic": None, "ms": stage_ms["m2l"],
                    "algorithmic": f"{nm2l} M2L pairs x 2K^2 flops, K=(p+1)^2={K}",
                    "peak_source": fp64_src if prec in (0, 1) else fp32_src})
    return out


def pass_rooflines(stage_ms: dict, ex, prec: int, info, n: int):
    """The up- and downward passes against HBM, with the algorithmic bytes of
    each (b = bytes per real coefficient, K = (p+1)^2 real coefficients, L =
    leaves): P2M 16N + L K b, M2M sum over internal cells of (children + 1) K b,
    L2L 3 K b per non-root cell, L2P 16N + L K b + 16N.  Times are the stage
    events inside the timed region (latency-bound stages: small fractions)."""
    pk, _ = peaks()
    hbm = float(pk["hbm_gbs"])
    K = (P + 1) ** 2
    b = 8 if prec in (0, 1) else 4
    cc = ex["child_count"]
    nleaf = int((cc == 0).sum())
    internal = cc > 0
    ncell = len(cc)
    algo = {"p2m": 16 * n + nleaf * K * b,
            "m2m": int(((cc[internal] + 1) * K * b).sum()),
            "l2l": 3 * K * b * (ncell - 1),
            "l2p": 16 * n + nleaf * K * b + 16 * n}
    out = []
    for name, bytes_ in algo.items():
        if name in stage_ms and stage_ms[name] > 0:
            gbs = bytes_ / (stage_ms[name] * 1e-3) / 1e9
            out.append({"stage": name, "bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                        "frac": gbs / hbm, "bytes": int(bytes_), "ms": stage_ms[name]})
    return out


def fp64_roofline_ratio(value: float, n: int, ex, v64):
    """The headline against the plain FP64 GPU path as it would run at its
    FP64-pipe roofline: the FP64 evaluation's algorithmic flops (M2L pairs x 2K^2
    + P2P pairs x 20) at the measured FP64 FMA rate, the tree build free.  A
    ratio against an ideal denominator (the measured one is vs_fp64_gpu_path)."""
    if not v64:
        return None
    K = (P + 1) ** 2
    flops = len(ex["m2l"]) * 2.0 * K * K + p2p_pairs(ex) * float(P2P_FLOPS_PER_PAIR)
    ideal_s = flops / (FP64_TFLOPS_MEASURED * 1e12)
    return {"ratio": value / (n / ideal_s), "fp64_ideal_ms": ideal_s * 1e3,
            "fp64_measured_ms": v64["ms_per_step"],
            "fp64_frac_of_roofline": ideal_s * 1e3 / v64["ms_per_step"]}


def use_mutual(args) -> bool:
    """The mutual near field applies to the FP32 near field of the stage-by-stage
    evaluation (the task graph and the FP64 path keep the non-mutual form)."""
    return args.mutual and args.precision != 0 and not args.task_graph


def execution_name(args) -> str:
    if use_mutual(args):
        return "staged kernels, mutual near field"
    if args.staged:
        return "staged kernels"
    if args.precision == 3:
        return "persistent task graph (one launch)" if args.task_graph else "staged kernels"
    return "persistent task queue"


def schedule_variant(fmm, torch, pos, q, phi64, f64, flush, stream, flags: int, steps: int = 3):
    """The same system and precision under the other schedule of the mixed form
    (the persistent task graph, or the staged kernels): build + evaluation
    particles/s, the evaluation alone, and the error against the FP64 GPU path."""
    n = pos.shape[0]
    phi = torch.empty_like(phi64)
    force = torch.empty_like(f64)
    ts, te = [], []
    for k in range(steps + 2):
        flush.zero_()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        t = fmm.build_tree(pos, p=P, leaf_size=LEAF, theta=THETA, precision=3, flags=flags)
        e1.record(stream)
        t.evaluate(q, phi=phi, force=force)
        e2.record(stream)
        torch.cuda.synchronize()
        status = t.status()
        t.close()
        if status != fmm.FMM_OK:
            return {"error": f"status {status}"}
        if k >= 2:
            ts.append(e0.elapsed_time(e2))
            te.append(e1.elapsed_time(e2))
    ms = statistics.median(ts)
    return {"execution": "persistent task graph (one launch)" if flags & fmm.TASK_GRAPH else "staged kernels",
            "value": n / (ms * 1e-3), "ms_per_step": ms, "evaluate_ms": statistics.median(te), "steps": steps,
            "dtype": PREC_DTYPE[3],
            "rel_l2_vs_fp64_gpu": {"phi": float(((phi - phi64).norm() / phi64.norm()).item()),
                                   "force": float(((force - f64).norm() / f64.norm()).item())}}


def p2p_form_variant(fmm, torch, pos, q, phi64, f64, flush, stream, ex, mutual: bool, iso_p2p_ms, steps: int = 3):
    """The mixed form with the other near-field form on the same system: the
    mutual one (FMM_MUTUAL, paper Section 4: each cross-leaf pair evaluated once
    for both leaves) or the non-mutual one (each leaf's sums by its own work
    items).  Build + evaluation particles/s, the evaluation alone, the near-field
    stage alone (FMM_NO_OVERLAP) beside the headline form's stage timed the same
    way, and the error against the FP64 GPU path.  Pair rates count directed
    pairs, the same algorithmic work in both forms."""
    n = pos.shape[0]
    phi = torch.empty_like(phi64)
    force = torch.empty_like(f64)
    ts, te, tp = [], [], []
    for k in range(2 * steps + 2):
        isolated = k >= steps + 1
        flush.zero_()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        t = fmm.build_tree(pos, p=P, leaf_size=LEAF, theta=THETA, precision=3,
                           flags=(fmm.MUTUAL if mutual else 0) | fmm.TIMING | (fmm.NO_OVERLAP if isolated else 0))
        e1.record(stream)
        t.evaluate(q, phi=phi, force=force)
        e2.record(stream)
        torch.cuda.synchronize()
        status = t.status()
        stages = t.stage_times()
        t.close()
        if status != fmm.FMM_OK:
            return {"error": f"status {status}"}
        if isolated:
            if k > steps + 1:
                tp.append(stages.get("p2p", 0.0))
        elif k >= 1:
            ts.append(e0.elapsed_time(e2))
            te.append(e1.elapsed_time(e2))
    ms = statistics.median(ts)
    pairs = p2p_pairs(ex)
    p2p_ms = statistics.median(tp)
    out = {"execution": "staged kernels" + (", mutual near field" if mutual else ""), "value": n / (ms * 1e-3),
           "ms_per_step": ms, "evaluate_ms": statistics.median(te), "steps": steps, "dtype": PREC_DTYPE[3],
           "p2p_stage_ms_isolated": p2p_ms, "p2p_pairs_per_s_isolated": pairs / (p2p_ms * 1e-3),
           "rel_l2_vs_fp64_gpu": {"phi": float(((phi - phi64).norm() / phi64.norm()).item()),
                                  "force": float(((force - f64).norm() / f64.norm()).item())}}
    if iso_p2p_ms:
        out["headline_p2p_stage_ms_isolated"] = iso_p2p_ms
        out["headline_p2p_pairs_per_s_isolated"] = pairs / (iso_p2p_ms * 1e-3)
    return out


def uvwx_variant(fmm, torch, pos, q, phi64, f64, flush, stream, flags: int, steps: int = 3):
    """The mixed form on the same system with the lists built from the
    parent-neighbour-child relationship (FMM_LISTS_UVWX, paper Section 2.1:
    V lists by M2L, U and the W / X leaves by direct sums) instead of the
    size/distance test: particles/s of build + evaluation, the list sizes, and
    the error against the plain FP64 GPU path (a different FMM of the same
    sum: the difference is both methods' truncation error)."""
    n = pos.shape[0]
    phi = torch.empty_like(phi64)
    force = torch.empty_like(f64)
    ts, te = [], []
    info = None
    for k in range(steps + 1):
        flush.zero_()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        t = fmm.build_tree(pos, p=P, leaf_size=LEAF, theta=THETA, precision=3, flags=flags | fmm.LISTS_UVWX)
        e1.record(stream)
        t.evaluate(q, phi=phi, force=force)
        e2.record(stream)
        torch.cuda.synchronize()
        status = t.status()
        info = t.info()
        t.close()
        if status != fmm.FMM_OK:
            return {"error": f"status {status}"}
        if k >= 1:
            ts.append(e0.elapsed_time(e2))
            te.append(e1.elapsed_time(e2))
    ms = statistics.median(ts)
    return {"execution": "staged kernels" + (", mutual near field" if flags & fmm.MUTUAL else ""),
            "lists": "parent-neighbour-child (U/V/W/X, W and X as direct sums)",
            "value": n / (ms * 1e-3), "ms_per_step": ms, "evaluate_ms": statistics.median(te), "steps": steps,
            "dtype": PREC_DTYPE[3], "nm2l": int(info.nm2l), "np2p": int(info.np2p),
            "rel_l2_vs_fp64_gpu": {"phi": float(((phi - phi64).norm() / phi64.norm()).item()),
                                   "force": float(((force - f64).norm() / f64.norm()).item())}}


def plummer_variant(fmm, torch, dev, flush, stream, steps: int = 3):
    """The mixed form on the Plummer configuration (1M particles, p = 8, leaf 64,
    theta = 0.4): particles/s of build + evaluation and its error against the
    plain FP64 GPU path on the same system."""
    import workloads as W
    _, n0, p, leaf, theta = SYSTEMS["plummer"]
    wl = W.make_workload("plummer")
    pos = torch.tensor(wl.pos, dtype=torch.float64, device=dev)
    q = torch.tensor(wl.q, dtype=torch.float64, device=dev)
    t64 = fmm.build_tree(pos, p=p, leaf_size=leaf, theta=theta, precision=fmm.PREC_FP64)
    phi64, f64 = t64.evaluate(q)
    t64.close()
    phi = torch.empty_like(phi64)
    force = torch.empty_like(f64)
    ts = []
    for k in range(steps + 2):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        t = fmm.build_tree(pos, p=p, leaf_size=leaf, theta=theta, precision=fmm.PREC_MIXED_TC)
        t.evaluate(q, phi=phi, force=force)
        e1.record(stream)
        torch.cuda.synchronize()
        t.close()
        if k >= 2:
            ts.append(e0.elapsed_time(e1))
    ms = statistics.median(ts)
    return {"workload": f"{SYSTEMS['plummer'][0]}, N={wl.n}, p={p}, leaf={leaf}, theta={theta}",
            "value": wl.n / (ms * 1e-3), "ms_per_step": ms, "steps": steps, "dtype": PREC_DTYPE[3],
            "rel_l2_vs_fp64_gpu": {"phi": float(((phi - phi64).norm() / phi64.norm()).item()),
                                   "force": float(((force - f64).norm() / f64.norm()).item())}}


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_1203_0889_gb300 as fmm
    import workloads as W

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    stream = torch.cuda.current_stream()
    wl = W.make_workload(WORKLOAD, n=args.n, seed=workload_seed(rank))
    n = wl.n
    pos = torch.tensor(wl.pos, dtype=torch.float64, device=dev)
    q = torch.tensor(wl.q, dtype=torch.float64, device=dev)
    phi = torch.empty(n, dtype=torch.float64, device=dev)
    force = torch.empty((n, 3), dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    flags = fmm.TIMING | (fmm.STAGED if args.staged else 0) | (fmm.TASK_GRAPH if args.task_graph else 0) | \
        (fmm.MUTUAL if use_mutual(args) else 0)

    def step():
        t = fmm.build_tree(pos, p=P, leaf_size=LEAF, theta=THETA, precision=args.precision, flags=flags)
        t.evaluate(q, phi=phi, force=force)
        return t

    # accuracy of this path against the plain FP64 GPU path (outside the timed region)
    t64 = fmm.build_tree(pos, p=P, leaf_size=LEAF, theta=THETA, precision=fmm.PREC_FP64)
    phi64, f64 = t64.evaluate(q)
    torch.cuda.synchronize()
    t64.close()
    tt = step()
    torch.cuda.synchronize()
    ex = tt.export()
    info = tt.info()
    tt.close()
    err_phi = float(((phi - phi64).norm() / phi64.norm()).item())
    err_f = float(((force - f64).norm() / f64.norm()).item())

    for _ in range(args.warmup):
        step().close()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stage_acc = {}
    launches = 0
    wall0 = time.perf_counter()
    ev_mid = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.zero_()                       # evict L2 between steps (outside the event pair)
        ev[k][0].record(stream)
        t = fmm.build_tree(pos, p=P, leaf_size=LEAF, theta=THETA, precision=args.precision, flags=flags)
        ev_mid[k].record(stream)            # build | evaluate
        t.evaluate(q, phi=phi, force=force)
        ev[k][1].record(stream)
        for name, ms in t.stage_times().items():
            stage_acc[name] = stage_acc.get(name, 0.0) + ms
        launches += t.kernel_launches(build=True) + t.kernel_launches(build=False)
        t.close()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    wall = time.perf_counter() - wall0
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    build_ms = statistics.median(a.elapsed_time(m) for (a, _), m in zip(ev, ev_mid))
    eval_ms = statistics.median(m.elapsed_time(b) for (_, b), m in zip(ev, ev_mid))
    total_s = sum(step_ms) * 1e-3
    total_s = max_over_ranks(total_s, dev)
    value = job_throughput(n, world, args.steps, total_s)
    stage_ms = {k: v / args.steps for k, v in stage_acc.items()}
    props = torch.cuda.get_device_properties(dev)
    roofs = kernel_rooflines(stage_ms, ex, args.precision, props.multi_processor_count, info, use_mutual(args))
    roof = max(roofs, key=lambda r: r["ms"]) if roofs else None
    passes = pass_rooflines(stage_ms, ex, args.precision, info, n)
    for r in roofs:
        if r["kernel"] in ("k_p2p", "k_p2p_mutual"):
            # the same pairs against the reciprocal-square-root (MUFU) bound, and both
            # bounds at the median SM clock seen under load
            f_load = clocks.get("sm_mhz") or 2070.0
            pairs = p2p_pairs(ex)
            nsm = props.multi_processor_count
            r["mufu_bound_pairs_per_s"] = nsm * 16 * 2070e6
            r["pairs_per_s"] = pairs / (r["ms"] * 1e-3)
            r["frac_at_loaded_clock"] = r["achieved"] / (r["peak"] * f_load / 2070.0)
            r["loaded_sm_mhz"] = f_load
    # the same kernels with nothing running beside them (FMM_NO_OVERLAP: P2P and
    # the far field one after the other), outside the timed region: the step
    # overlaps P2P with the far field, which stretches both kernels' event times
    iso_acc = {}
    if (args.precision == 3 and not args.task_graph) or args.staged or use_mutual(args):
        for k in range(4):
            flush.zero_()
            ti = fmm.build_tree(pos, p=P, leaf_size=LEAF, theta=THETA, precision=args.precision,
                                flags=flags | fmm.NO_OVERLAP)
            ti.evaluate(q, phi=phi, force=force)
            torch.cuda.synchronize()
            if k > 0:
                for name, ms in ti.stage_times().items():
                    iso_acc[name] = iso_acc.get(name, 0.0) + ms / 3
            ti.close()
        iso = {r["kernel"]: r for r in kernel_rooflines(iso_acc, ex, args.precision, props.multi_processor_count,
                                                         info, use_mutual(args))}
        for r in roofs:
            if r["kernel"] in iso:
                r["isolated"] = {k: iso[r["kernel"]][k] for k in ("ms", "achieved", "frac")}
        # the dominant kernel is the one with the most work, i.e. the longest time
        # alone (inside the step P2P is stretched by the far field beside it); its
        # share agrees with the serialised ncu launch list
        if roofs:
            roof = max(roofs, key=lambda r: r.get("isolated", {}).get("ms", r["ms"]))

    # the other precisions on the same system, a few steps each (context for the
    # headline: the plain FP64 GPU path is the accuracy reference)
    variants = {}
    if not args.no_variants:
        for vp in (0, 1, 2):
            if vp == args.precision:
                continue
            vsteps = 2 if vp in (0, 1) else 3
            step_v = lambda: fmm.build_tree(pos, p=P, leaf_size=LEAF, theta=THETA, precision=vp,  # noqa: E731
                                            flags=fmm.TIMING)
            tv = step_v()
            pv, fv = tv.evaluate(q)
            tv.close()
            torch.cuda.synchronize()
            ms = 0.0
            vstage = {}
            for _ in range(vsteps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                tv = step_v()
                tv.evaluate(q, phi=phi, force=force)
                e1.record(stream)
                torch.cuda.synchronize()
                ms += e0.elapsed_time(e1) / vsteps
                for name, sms in tv.stage_times().items():
                    vstage[name] = vstage.get(name, 0.0) + sms / vsteps
                vinfo = tv.info()
                tv.close()
            vroofs = kernel_rooflines(vstage, ex, vp, props.multi_processor_count, vinfo)
            variants[PREC_NAMES[vp]] = {
                "value": n / (ms * 1e-3), "ms_per_step": ms, "steps": vsteps, "dtype": PREC_DTYPE[vp],
                "rel_l2_vs_fp64_gpu": {"phi": float(((pv - phi64).norm() / phi64.norm()).item()),
                                       "force": float(((fv - f64).norm() / f64.norm()).item())},
                "roofline": max(vroofs, key=lambda r: r["ms"]) if vroofs else None,
                "stage_ms": {k: round(v, 4) for k, v in vstage.items()}}
            del pv, fv
        if WORKLOAD != "plummer":
            variants["plummer_mixed_tc"] = plummer_variant(fmm, torch, dev, flush, stream)
        if args.precision == 3:
            variants["task_graph" if not args.task_graph else "staged"] = schedule_variant(
                fmm, torch, pos, q, phi64, f64, flush, stream, 0 if args.task_graph else fmm.TASK_GRAPH)
            if not args.task_graph:
                other = not use_mutual(args)
                variants["mutual_p2p" if other else "non_mutual_p2p"] = p2p_form_variant(
                    fmm, torch, pos, q, phi64, f64, flush, stream, ex, other, iso_acc.get("p2p"))

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        hpos = torch.tensor(wl.pos, dtype=torch.float64).pin_memory()
        hq = torch.tensor(wl.q, dtype=torch.float64).pin_memory()
        hphi = torch.empty(n, dtype=torch.float64).pin_memory()
        hforce = torch.empty((n, 3), dtype=torch.float64).pin_memory()

        def e2e_step():
            dpos = hpos.to(dev, non_blocking=True)
            dq = hq.to(dev, non_blocking=True)
            t = fmm.build_tree(dpos, p=P, leaf_size=LEAF, theta=THETA, precision=args.precision,
                               flags=flags & ~fmm.TIMING)
            ph, fo = t.evaluate(dq)
            hphi.copy_(ph, non_blocking=True)
            hforce.copy_(fo, non_blocking=True)
            return t

        for _ in range(2):
            e2e_step().close()
        torch.cuda.synchronize()
        ks = max(3, args.steps // 2)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tot = 0.0
        for _ in range(ks):
            flush.zero_()
            e0.record(stream)
            t = e2e_step()
            e1.record(stream)
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1) * 1e-3
            t.close()
        e2e = {"value": n * ks / tot, "unit": "particles/s", "h2d_bytes_per_step": n * 3 * 8 + n * 8,
               "d2h_bytes_per_step": n * 8 + n * 3 * 8}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.cpu_sample_n)

    # the parent-neighbour-child lists on the same system, after every other leg
    # (an error there is reported in the variant and leaves the rest measured)
    if not args.no_variants and args.precision == 3:
        try:
            variants["uvwx_lists"] = uvwx_variant(fmm, torch, pos, q, phi64, f64, flush, stream,
                                                  fmm.MUTUAL if use_mutual(args) else 0)
        except Exception as exc:   # noqa: BLE001
            variants["uvwx_lists"] = {"error": f"{type(exc).__name__}: {exc}"[:300]}

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "particles/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_s * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": PREC_DTYPE[args.precision], "data": "synthetic",
            "config": {"workload": workload_line(n),
                       "step": "fmm_build_tree + fmm_evaluate (potentials and forces)",
                       "precision": PREC_NAMES[args.precision], "l2": "flushed between steps (512 MB write)",
                       "execution": execution_name(args),
                       "parallelism": f"replicas x{world}", "ncell": info.ncell, "nleaf": info.nleaf,
                       "nm2l": info.nm2l, "np2p": info.np2p, "tc_pairs": info.tc_pairs,
                       "tc_classes": info.tc_classes,
                       "rel_l2_vs_fp64_gpu": {"phi": err_phi, "force": err_f},
                       "stage_ms": {k: round(v, 4) for k, v in stage_ms.items()},
                       "evaluate_ms": round(sum(v for k, v in stage_ms.items()
                                                if k in ("prepare", "p2p", "p2m", "m2m", "m2l", "l2l", "l2p",
                                                         "queue")), 4),
                       "wall_s": wall},
            "roofline": roof, "rooflines": roofs, "passes": passes, "variants": variants, "cpu_baseline": cpu,
            "e2e": e2e,
            "build_ms_per_step": build_ms, "evaluate_ms_per_step": eval_ms,
            "evaluate_particles_per_s": n / (eval_ms * 1e-3),
            "vs_fp64_gpu_path": (value / variants["fp64"]["value"]) if "fp64" in variants else None,
            "vs_fp64_roofline": fp64_roofline_ratio(value, n, ex, variants.get("fp64")),
            "gpu_launches": launches, "clocks": clocks,
        }
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------- CPU oracle

def cpu_baseline(sample_n: int):
    """The FP64 oracle as it stands (tree build + full FMM) on the host cores, on a
    smaller system of the bench workload's recipe; particles/s of that sample."""
    import oracle
    import workloads as W
    cores = os.cpu_count() or 1
    wl = W.make_workload(WORKLOAD, n=sample_n)
    t0 = time.perf_counter()
    T = oracle.build_tree(wl.pos, LEAF, THETA)
    T.evaluate(P, wl.q, nthreads=cores)
    dt = time.perf_counter() - t0
    return {"value": sample_n / dt, "unit": "particles/s", "cores": cores, "kind": "oracle",
            "sample": f"oracle tree build + FP64 FMM of a {WORKLOAD} system of N={sample_n} "
                      f"(same recipe, p={P}, leaf={LEAF}, theta={THETA}), {dt:.2f} s"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    import workloads as W
    oracle.build()
    cores = os.cpu_count() or 1
    n = min(args.cpu_sample_n, 1 << 16)
    wl = W.make_workload(WORKLOAD, n=n)

    def step():
        T = oracle.build_tree(wl.pos, LEAF, THETA)
        T.evaluate(P, wl.q, nthreads=cores)

    for _ in range(args.warmup):
        step()
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        step()
        ts.append(time.perf_counter() - t0)
    tot = sum(ts)
    value = n * args.steps / tot
    sample = (f"oracle tree build + FP64 FMM per step on a {WORKLOAD} system of N={n} (same recipe, p={P}, "
              f"leaf={LEAF}, theta={THETA})")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "particles/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_line(N_DEFAULT), "sample_n": n},
        "cpu_baseline": {"value": value, "unit": "particles/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "particles/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_batched(args):
    """512 independent systems (uniform / Plummer / clustered by index mod 3,
    N_s log-uniform in [1024, 65536], q ~ U[-1,1], p = 6, theta = 0.5, FP32):
    one batched tree, one task-queue evaluation replayed from a CUDA graph.
    The leaf size is picked by the autotuner on the first 64 systems."""
    import torch

    import paper_1203_0889_gb300 as fmm
    import workloads as W

    dev = torch.device("cuda", 0)
    systems = W.make_batched(512)
    sizes = np.array([len(s[1]) for s in systems], np.int64)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    pos = torch.tensor(np.concatenate([s[0] for s in systems]), dtype=torch.float64, device=dev)
    q = torch.tensor(np.concatenate([s[1] for s in systems]), dtype=torch.float32, device=dev)
    n = int(off[-1])
    k = 64
    leaf, tune = fmm.autotune_leaf_size(pos[:off[k]], q[:off[k]], offsets=off[:k + 1], repeats=2, p=6, theta=0.5,
                                        precision=fmm.PREC_FP32,
                                        candidates=(32, 48, 64, 96, 128, 192, 256, 384))
    prm = dict(p=6, leaf_size=leaf, theta=0.5, precision=fmm.PREC_FP32)
    phi = torch.empty(n, dtype=torch.float32, device=dev)
    force = torch.empty((n, 3), dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        t = fmm.build_tree_batched(pos, off, **prm)
        t.evaluate(q, phi=phi, force=force)
        t.close()
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(0.3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k_ in range(args.steps):
        flush.zero_()
        ev[k_][0].record()
        t = fmm.build_tree_batched(pos, off, **prm)
        t.evaluate(q, phi=phi, force=force)
        ev[k_][1].record()
        if k_ < args.steps - 1:
            t.close()
    torch.cuda.synchronize()
    total_s = sum(a.elapsed_time(b) for a, b in ev) * 1e-3
    g = fmm.capture_graph(t, q, phi, force)
    gt = []
    for _ in range(max(3, args.steps)):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g.replay()
        e1.record()
        torch.cuda.synchronize()
        gt.append(e0.elapsed_time(e1))
    clocks = sampler.stop()
    info = t.info()
    # the mixed tensor-core form on the same systems (stage-by-stage, not the
    # queue): context for the configuration's FP32 queue form
    mixed = None
    prm_m = dict(prm, precision=fmm.PREC_MIXED_TC)
    ts = []
    for k_ in range(args.warmup + args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        tm = fmm.build_tree_batched(pos, off, **prm_m)
        pm, fm = tm.evaluate(q)
        e1.record()
        torch.cuda.synchronize()
        if k_ >= args.warmup:
            ts.append(e0.elapsed_time(e1))
        tm.close()
    mixed = {"value": n / (statistics.median(ts) * 1e-3), "ms_per_step": statistics.median(ts),
             "rel_l2_vs_fp32_queue": {"phi": float(((pm - phi).norm() / phi.norm()).item()),
                                      "force": float(((fm - force).norm() / force.norm()).item())}}
    out = {
        "metric": METRIC, "value": n * args.steps / total_s, "unit": "particles/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_s * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"batched: 512 systems, N={n} in total (1024..65536 each), p=6, theta=0.5",
                   "step": "fmm_build_tree_batched + fmm_evaluate_batched", "leaf_size": leaf,
                   "autotune_ms": tune, "evaluate_graph_replay_ms": statistics.median(gt),
                   "evaluate_particles_per_s": n / (statistics.median(gt) * 1e-3),
                   "ncell": info.ncell, "nm2l": info.nm2l, "np2p": info.np2p,
                   "l2": "flushed between steps (512 MB write)"},
        "clocks": clocks, "gpu_launches": t.kernel_launches(build=True) + t.kernel_launches(build=False),
        "variants": {"mixed_tc": mixed},
    }
    print(json.dumps(out), flush=True)


def run_table(args):
    """Every configuration of the workload set on this GPU: throughput of the
    FP64 and reduced-precision forms (tree build + evaluation per step), their
    error against the FP64 oracle on sampled leaves, and the oracle itself on
    the host cores (bounded samples of the same recipes).  One JSON line plus a
    markdown table on stderr."""
    import torch

    import oracle
    import paper_1203_0889_gb300 as fmm
    import workloads as W

    oracle.build()
    dev = torch.device("cuda", 0)
    cores = os.cpu_count() or 1
    out = {"table": [], "cores": cores}

    def gpu_rate(pos, q, prec, p, leaf, theta, steps):
        res = None
        for k in range(steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            t = fmm.build_tree(pos, p=p, leaf_size=leaf, theta=theta, precision=prec)
            phi, f = t.evaluate(q)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            t.close()
            if k == 0:
                res = (phi.double().cpu().numpy(), f.double().cpu().numpy(), [])
            else:
                res[2].append(dt)
        return res[0], res[1], statistics.median(res[2])

    def cpu_rate(name, n, threads):
        wl = W.make_workload(name, n=n)
        t0 = time.perf_counter()
        T = oracle.build_tree(wl.pos, wl.leaf_size, wl.theta)
        T.evaluate(wl.p, wl.q, nthreads=threads)
        return n / (time.perf_counter() - t0)

    for name in ("uniform", "plummer", "clustered", "gradient"):
        wl = W.make_workload(name)
        n, p, leaf, theta = wl.n, wl.p, wl.leaf_size, wl.theta
        T = oracle.Tree(wl.pos, leaf, theta)
        leaves = np.nonzero(T.is_leaf)[0]
        pick = np.random.default_rng(1203).choice(leaves, size=min(64, len(leaves)), replace=False)
        idx, phi_ref, grad_ref = T.evaluate_leaves(p, wl.q, np.sort(pick))
        f_ref = -wl.q[idx, None] * grad_ref
        pos = torch.tensor(wl.pos, dtype=torch.float64, device=dev)
        q = torch.tensor(wl.q, dtype=torch.float64, device=dev)
        row = {"config": name, "n": n, "p": p, "leaf": leaf, "theta": theta, "sampled_particles": int(len(idx))}
        for prec in (0, 2, 3):
            phi, f, dt = gpu_rate(pos, q, prec, p, leaf, theta, steps=2 if prec == 0 else 3)
            if prec == 0:
                row["_phi64"], row["_f64"] = phi, f
            row[PREC_NAMES[prec]] = {
                "particles_per_s": n / dt, "ms_per_step": dt * 1e3,
                "rel_l2_vs_oracle": {"phi": float(np.linalg.norm(phi[idx] - phi_ref) / np.linalg.norm(phi_ref)),
                                     "force": float(np.linalg.norm(f[idx] - f_ref) / np.linalg.norm(f_ref))}}
        del T
        row["oracle_all_cores"] = cpu_rate(name, min(n, 1 << 17), cores)
        row["oracle_1_core"] = cpu_rate(name, min(n, 1 << 14), 1)
        # the oracle's direct sum (one core): all targets at N <= 16384, else 4096
        # seeded targets against all sources, extrapolated to N targets
        nt = min(n, 4096) if n > 16384 else n
        tg = np.sort(np.random.default_rng(4096).choice(n, size=nt, replace=False)) if nt < n else np.arange(n)
        t0 = time.perf_counter()
        ph_d, gr_d = oracle.direct_targets(wl.pos, wl.q, tg)
        dt_d = (time.perf_counter() - t0) * n / nt
        row["oracle_direct_1_core_particles_per_s"] = n / dt_d
        # the mixed form against the exact sum on those targets (FMM truncation included)
        phi_m, f_m, _ = gpu_rate(pos, q, 3, p, leaf, theta, steps=1)
        f_d = -wl.q[tg, None] * gr_d
        row["mixed_tc"]["rel_l2_vs_direct_sum"] = {
            "phi": float(np.linalg.norm(phi_m[tg] - ph_d) / np.linalg.norm(ph_d)),
            "force": float(np.linalg.norm(f_m[tg] - f_d) / np.linalg.norm(f_d))}
        row["fp64"]["rel_l2_vs_direct_sum"] = {
            "phi": float(np.linalg.norm(row.pop("_phi64")[tg] - ph_d) / np.linalg.norm(ph_d)),
            "force": float(np.linalg.norm(row.pop("_f64")[tg] - f_d) / np.linalg.norm(f_d))}
        if name == "gradient":
            # forward + backward through the autograd node (FP32), L = sum w phi
            fn = fmm.FMMFunction
            w = torch.tensor(wl.extra["w"], dtype=torch.float32, device=dev)
            pos32 = pos.clone().requires_grad_(True)
            q32 = q.float().requires_grad_(True)
            ts = []
            for k in range(4):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                t = fmm.build_tree(pos32.detach(), p=p, leaf_size=leaf, theta=theta, precision=fmm.PREC_FP32,
                                   flags=fmm.OUT_FIELD)
                loss = (fn.apply(pos32, q32, t) * w).sum()
                loss.backward()
                torch.cuda.synchronize()
                ts.append(time.perf_counter() - t0)
                t.close()
                pos32.grad = None
                q32.grad = None
            row["forward_backward_fp32_particles_per_s"] = n / statistics.median(ts[1:])
        out["table"].append(row)
        print(json.dumps(row), file=sys.stderr, flush=True)
    # batched systems (FP32, task queue), build + evaluate per step
    systems = W.make_batched(512)
    sizes = np.array([len(s_[1]) for s_ in systems], np.int64)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    pos = torch.tensor(np.concatenate([s_[0] for s_ in systems]), dtype=torch.float64, device=dev)
    q = torch.tensor(np.concatenate([s_[1] for s_ in systems]), dtype=torch.float32, device=dev)
    leaf_b, _ = fmm.autotune_leaf_size(pos[:off[64]], q[:off[64]], offsets=off[:65], repeats=2, p=6, theta=0.5,
                                       precision=fmm.PREC_FP32, candidates=(32, 48, 64, 96, 128, 192, 256, 384))
    rates = {}
    for prec in (fmm.PREC_FP32, fmm.PREC_MIXED_TC):
        ts = []
        for k in range(4):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            t = fmm.build_tree_batched(pos, off, p=6, leaf_size=leaf_b, theta=0.5, precision=prec)
            t.evaluate(q)
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
            t.close()
        rates[PREC_NAMES[prec]] = {"particles_per_s": int(off[-1]) / statistics.median(ts[1:])}
    out["table"].append({"config": "batched", "n": int(off[-1]), "systems": 512, "p": 6, "leaf": leaf_b, **rates})
    print(json.dumps(out), flush=True)
    lines = ["| config | N | GPU FP64 p/s | GPU FP32 p/s | GPU mixed p/s | error FP64 / FP32 / mixed (phi, F) vs oracle "
             f"| oracle {cores} cores p/s | oracle 1 core p/s |", "|---|---|---|---|---|---|---|---|"]
    for r in out["table"]:
        if r["config"] == "batched":
            lines.append(f"| batched 512 (leaf {r['leaf']}) | {r['n']} | | {r['fp32']['particles_per_s']:.3g} | "
                         f"{r['mixed_tc']['particles_per_s']:.3g} | | | |")
            continue
        e = " / ".join(f"{r[k]['rel_l2_vs_oracle']['phi']:.1e}, {r[k]['rel_l2_vs_oracle']['force']:.1e}"
                       for k in ("fp64", "fp32", "mixed_tc"))
        lines.append(f"| {r['config']} | {r['n']} | {r['fp64']['particles_per_s']:.3g} | "
                     f"{r['fp32']['particles_per_s']:.3g} | {r['mixed_tc']['particles_per_s']:.3g} | {e} | "
                     f"{r['oracle_all_cores']:.3g} | {r['oracle_1_core']:.3g} |")
    print("\n".join(lines), file=sys.stderr, flush=True)


def run_granularity(args):
    """Task granularity against problem size (the paper's queue threshold Q
    versus N study, on the device queue): uniform particles, p = 6 and 9,
    N = 1e5, 1e6, 1e7, leaf sizes 16..256; FP32 task-queue evaluation (one
    persistent launch running the task DAG).  A leaf size fixes the number of
    tasks (cells and leaves, about N / leaf each), so the sweep shows where
    per-task scheduling stops being amortised.  Prints one JSON line."""
    import torch

    import paper_1203_0889_gb300 as fmm
    import workloads as W

    dev = torch.device("cuda", 0)
    rows = []
    ints = lambda s: [int(v) for v in s.split(",") if v]  # noqa: E731
    for n in ints(args.granularity_n):
        wl = W.make_workload("uniform", n=n, seed=12030889 * 10 + 6)
        pos = torch.tensor(wl.pos, dtype=torch.float64, device=dev)
        q = torch.tensor(wl.q, dtype=torch.float32, device=dev)
        for p in ints(args.granularity_p):
            for leaf in ints(args.granularity_leaf):
                t = fmm.build_tree(pos, p=p, leaf_size=leaf, theta=0.5, precision=fmm.PREC_FP32)
                info = t.info()
                t.evaluate(q)
                torch.cuda.synchronize()
                ts = []
                for _ in range(3):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    t.evaluate(q)
                    e1.record()
                    torch.cuda.synchronize()
                    ts.append(e0.elapsed_time(e1))
                ms = statistics.median(ts)
                ntask = info.ncell + 2 * info.nleaf   # M2M/M2L/L2L per cell, P2M + P2P + L2P per leaf (P2M grouped)
                rows.append({"n": n, "p": p, "leaf": leaf, "ncell": info.ncell, "nleaf": info.nleaf,
                             "tasks": ntask, "n_over_tasks": n / ntask, "evaluate_ms": ms,
                             "particles_per_s": n / (ms * 1e-3), "us_per_task": ms * 1e3 / ntask,
                             "status": t.status()})
                t.close()
                print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    print(json.dumps({"study": "task granularity vs N (FP32 task queue, uniform, theta 0.5)", "rows": rows}),
          flush=True)


def main():
    args = parse()
    if args.workload in SYSTEMS:
        select_workload(args.workload)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "table":
        run_table(args)
    elif args.workload == "granularity":
        run_granularity(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
