#!/usr/bin/env python
"""Throughput of the exact DBSCAN hot path on GB300; prints one JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]

A step is one full clustering (prep, pair test + count -> core flags, union,
border, labels) of one synthetic instance already resident in HBM.  The
default run measures n = 500,000 points in d = 2 (50 Gaussian blobs with sigma
log-uniform in [0.002, 0.02] plus 20% noise, eps = 0.005, min_pts = 10), which
runs on the eps-grid path, and adds compact records of the other workloads
(the same recipe in 3-D, the d = 64 precision form on FP16 and BF16 tensor
cores, the 4,096-instance batch and the served job stream) under
"subrecords".  --workload NAME prints the full record of one workload.

Metric: G pair-tests/s, the pair predicates D(p,q) <= T the device evaluated
(its per-pass counters, read after every timed step) per second.  Pairs the
method decides without a test (inside a clique cell of the eps-grid, after an
early exit) are not counted; the eps-grid's candidate pairs are reported
beside it.  The L2 is flushed (a 256 MiB write) before every timed step; each
step is timed with CUDA events on the plan's stream.  With N > 1 (torchrun)
every rank runs its own replica on its own GPU (the path does not shard) and
the value is the sum over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1506_02226_gb300 import inputs  # noqa: E402

WORKLOADS = {
    "lowd2": ("500k points, d=2, 50 blobs + 20% noise, eps=0.005, min_pts=10", lambda: inputs.large_lowd(2)),
    "lowd3": ("500k points, d=3, 50 blobs + 20% noise, eps=0.005, min_pts=10", lambda: inputs.large_lowd(3)),
    "small": ("2k points, d=2, 5 blobs + 10% noise, eps=0.02, min_pts=5", inputs.small_2d),
    "highd": ("200k points, d=64, 100 blobs + 15% noise, eps=median 30-NN distance, min_pts=20, FP16 tensor-core "
              "Gram pair test", inputs.high_d),
    "highd_bf16": ("200k points, d=64, as highd with BF16 tensor-core Gram pair test", inputs.high_d),
    "highd_simt": ("200k points, d=64, as highd with the exact CUDA-core pair test", inputs.high_d),
    "midd4": ("200k points, d=4, 50 blobs + 20% noise, eps=0.005*sqrt(d/2), min_pts=10, projected grid",
              lambda: inputs.mid_d(4)),
    "midd8": ("200k points, d=8, 50 blobs + 20% noise, eps=0.005*sqrt(d/2), min_pts=10, projected grid",
              lambda: inputs.mid_d(8)),
}
CPU_SAMPLE = {"lowd2": 200_000, "lowd3": 200_000, "small": 2000, "highd": 40_000, "highd_bf16": 40_000,
              "highd_simt": 40_000, "midd4": 100_000, "midd8": 100_000}
# workloads whose record also times the same instance on the all-pairs path
COMPARE_ALLPAIRS = {"midd4", "midd8"}
PRECISION = {"highd_bf16": 3, "highd_simt": 1}


def work_units(points: np.ndarray, eps: float, d: int) -> int:
    """Pair tests of one clustering: eps-grid candidate pairs for d <= 3, n^2 otherwise."""
    return grid_candidate_pairs(points, eps) if d <= 3 else points.shape[0] ** 2


# ------------------------------------------------------------------ work units
def grid_structure(points: np.ndarray, eps: float) -> dict:
    """The eps-grid of an instance, counted on the host with numpy.

    Cell side c = floor(sqrt(floor(T/d))) + 1 grid units; a point's candidates
    are the points of its own cell and of every occupied cell at an offset o
    with sum_k [o_k != 0]((|o_k|-1)c+1)^2 <= T.  Returns the ordered candidate
    pairs, the occupied cells and the neighbour-list entries (occupied cells at
    kept offsets, adjacent |o_k| <= 1 and outer ring separately).
    """
    u = np.rint(points.astype(np.float64) * 1024).astype(np.int64)
    n, d = u.shape
    e = float(np.float32(eps))
    T = min(math.floor(e * e * 1048576.0), d * 1023 * 1023)
    c, offs = grid_offsets(d, T)
    G = -(-1024 // c)
    cells = u // c
    key = np.zeros(n, np.int64)
    for k in reversed(range(d)):
        key = key * G + cells[:, k]
    uk, cnt = np.unique(key, return_counts=True)
    coords = np.stack([(uk // G ** k) % G for k in range(d)], axis=1)
    total = np.zeros(len(uk), np.int64)
    near = far = 0
    for off in offs:
        nc = coords + np.array(off)
        ok = np.all((nc >= 0) & (nc < G), axis=1)
        nk = np.zeros(len(uk), np.int64)
        for k in reversed(range(d)):
            nk = nk * G + nc[:, k]
        pos = np.clip(np.searchsorted(uk, nk), 0, len(uk) - 1)
        hit = ok & (uk[pos] == nk)
        total += np.where(hit, cnt[pos], 0)
        if max(abs(x) for x in off) <= 1:
            near += int(hit.sum())
        else:
            far += int(hit.sum())
    return {"candidate_pairs": int((cnt * (cnt + total)).sum()), "cells": len(uk), "near_entries": near,
            "far_entries": far}


def grid_candidate_pairs(points: np.ndarray, eps: float) -> int:
    """Ordered candidate pairs of the eps-grid (host-side count, numpy)."""
    return grid_structure(points, eps)["candidate_pairs"]


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = [l.split(", ") for l in out.strip().splitlines() if l.count(",") >= 8]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ roofline
def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return {"hbm_gbs": p["hbm_gbs"], "bf16_tflops": p["bf16_tflops"], "sm_max_mhz": p.get("sm_max_mhz", 2070.0),
                "src": "measured"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0, "src": "fallback"}


def grid_offsets(d: int, T: int):
    """Cell side and neighbour offsets of the eps-grid (same rule as the library)."""
    import itertools
    c = math.isqrt(T // d) + 1
    r = -(-math.isqrt(T) // c)
    offs = [o for o in itertools.product(range(-r, r + 1), repeat=d)
            if any(o) and sum(((abs(x) - 1) * c + 1) ** 2 for x in o if x) <= T]
    return c, offs


# DRAM bytes per launch of a dominant kernel from an ncu capture (profiles/), with
# the sha1 prefix of the kernel's source file when it was captured: a changed
# source means the counters no longer describe the kernel, and the bench line
# reports traffic null.
NCU_TRAFFIC = {
    ("lowd2", "grid_count"): (17419776, "paper_1506_02226_gb300/csrc/grid.cu", "faffd4840d06"),
    ("lowd2", "grid_union_near"): (10742272, "paper_1506_02226_gb300/csrc/grid.cu", "faffd4840d06"),
    ("lowd3", "grid_count"): (32878592, "paper_1506_02226_gb300/csrc/grid.cu", "faffd4840d06"),
    ("lowd3", "grid_union_near"): (23241728, "paper_1506_02226_gb300/csrc/grid.cu", "faffd4840d06"),
}


def ncu_traffic(workload: str, kernel: str):
    rec = NCU_TRAFFIC.get((workload, kernel))
    if rec is None:
        return None
    import hashlib
    nbytes, path, sha = rec
    try:
        with open(os.path.join(ROOT, path), "rb") as f:
            cur = hashlib.sha1(f.read()).hexdigest()
    except OSError:
        return None
    return nbytes if cur.startswith(sha) else None


def algorithmic_work(name: str, n: int, d: int, gs: dict | None):
    """(bound, bytes per launch) of a grid kernel: the bytes it has to move at
    least, counting every input it must read and every output it must write
    once.  gs is the instance's grid_structure (cells C, neighbour-list entries
    E = adjacent En + outer Ef; H hash slots).

      prep     reads x (4d), writes packed point (16) and hash slot (4), one
               hash entry (8)                                 (4d + 28) n
      cells    reads key and count of every slot (8), writes the packed
               {key, id} table (8), 24 per cell               16 H + 24 C
      scatter  reads slot, cell id and packed point (24), writes packed
               point, index and cell id (24), one cursor (4)  52 n
      nbrs     per cell key and list length (8), per entry a hash entry (8)
               and the list entry (4)                         8 C + 12 E
      count    per point the packed point (16), index (4), core flag and
               parent written (5); per cell 32 (range, length, rep, centre);
               per entry list entry and neighbour range (12)  25 n + 32 C + 12 E
      union    per cell 32; per adjacent entry list entry, key, rep and
               centre point (28); per outer entry 12           32 C + 28 En / 12 Ef
      border   per point core flag (1) and border written (4) 5 n
      root     per cell rep, parent and root (16)             16 C (also the snapshot
               taken between the adjacent and outer-ring merges)
      label    per point index, cell, flag, cell root, border (17), label (4)  21 n
    """
    if d > 3 or gs is None:
        return None, 0
    C, En, Ef = gs["cells"], gs["near_entries"], gs["far_entries"]
    E = En + Ef
    H = 1 << max(10, math.ceil(math.log2(2 * n)))
    table = {
        "grid_prep": (4 * d + 28) * n,
        "grid_cells": 16 * H + 24 * C,
        "grid_scatter": 52 * n,
        "grid_nbrs": 8 * C + 12 * E,
        "grid_count": 25 * n + 32 * C + 12 * E,
        "grid_union_near": 32 * C + 28 * En,
        "grid_union_far": 32 * C + 12 * Ef,
        "grid_border": 5 * n,
        "grid_cell_root": 16 * C,
        "grid_root_snapshot": 16 * C,
        "grid_label": 21 * n,
    }
    if name in table:
        return "hbm", table[name]
    return None, 0


def fp32_peak_tops():
    """FP32-pipe instruction peak of this GPU: SMs x 128 lanes x max SM clock."""
    import torch
    peaks = load_peaks()
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    return sms * 128 * peaks["sm_max_mhz"] * 1e6 / 1e12, sms


def pair_ops(d: int) -> int:
    """FP32-pipe instructions of one pair test: Gram form d+2 (d <= 16), direct form 2d+1."""
    return d + 2 if d <= 16 else 2 * d + 1


# ------------------------------------------------------------------ replicas
def max_over_ranks(local_ms: float, dist, device) -> float:
    """Largest per-rank time (the job finishes when its slowest replica does)."""
    import torch
    if dist is None:
        return local_ms
    t = torch.tensor([local_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, ms_per_step: float) -> float:
    """Units all replicas processed per second (weak scaling: each rank runs one replica)."""
    return world * units_per_rank / (ms_per_step * 1e-3)


# ------------------------------------------------------------------ arms
# Device counters 16..19 of a plan: pair tests of the count, merge, border and
# outer-ring merge passes; the kernels that evaluate pairs, by pass.
PASS_OF = {"grid_count": 0, "grid_union_near": 1, "grid_border": 2, "grid_union_far": 3,
           "ap_count": 0, "ap_union": 1, "ap_border": 2, "tc_count": 0, "tc_union": 1, "tc_border": 2,
           "mid_count": 0, "mid_union": 1, "mid_border": 2}


def run_reference(args, wl_name):
    """The oracle (plain CPU brute force) timed on bounded samples of the workload."""
    import oracle
    desc, make = WORKLOADS[wl_name]
    inst = make()
    cores = os.cpu_count() or 1
    # Size the per-step sample so that warm-up + timed steps take about two minutes
    # (brute force costs ~m^2): calibrate on a small subsample first.
    m0 = min(20_000, inst.n)
    cal = inputs.subsample(inst, m0, seed=999)
    t0 = time.perf_counter()
    oracle.dbscan(cal.points, cal.eps, cal.min_pts, nthreads=cores)
    t_cal = max(time.perf_counter() - t0, 1e-3)
    target = min(10.0, 120.0 / (args.warmup + args.steps))
    m = int(min(inst.n, max(2000, m0 * math.sqrt(target / t_cal))))
    times, units, pts = [], [], []
    for step in range(args.warmup + args.steps):
        sub = inputs.subsample(inst, m, seed=step)
        t0 = time.perf_counter()
        oracle.dbscan(sub.points, sub.eps, sub.min_pts, nthreads=cores)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
            units.append(sub.n * sub.n)  # brute force evaluates every ordered pair
            pts.append(sub.n)
    value = sum(units) / sum(times) / 1e9
    ms = 1e3 * sum(times) / len(times)
    sample = (f"oracle on {m}-point uniform subsamples of the {desc} workload, one per step; it evaluates all "
              f"m^2 ordered pairs")
    print(json.dumps({
        "impl": "reference", "metric": "G pair-tests/s", "value": value, "unit": "G pair-tests/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": wl_name + ": " + desc, "sample_points": m},
        "points_per_s": sum(pts) / sum(times),
        "cpu_baseline": {"value": value, "unit": "G pair-tests/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "G pair-tests/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def cpu_baseline(inst, wl_name, desc):
    """The oracle as it stands on a bounded subsample, all host cores and one thread.
    Brute force evaluates every ordered pair, so its rate is m^2 / time."""
    import oracle
    m = min(CPU_SAMPLE[wl_name], inst.n)
    sub = inputs.subsample(inst, m, seed=12345)
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    oracle.dbscan(sub.points, sub.eps, sub.min_pts, nthreads=cores)
    dt = time.perf_counter() - t0
    m1 = max(m // 4, min(m, 1000))
    sub1 = inputs.subsample(inst, m1, seed=12345)
    t1 = time.perf_counter()
    oracle.dbscan(sub1.points, sub1.eps, sub1.min_pts, nthreads=1)
    dt1 = time.perf_counter() - t1
    return {"value": m * m / dt / 1e9, "unit": "G pair-tests/s", "cores": cores, "kind": "oracle",
            "points_per_s": m / dt,
            "sample": f"full oracle run on a {m}-point uniform subsample of the {desc} workload "
                      f"({m * m} pair tests, all ordered pairs, {dt:.2f} s)",
            "single_thread": {"value": m1 * m1 / dt1 / 1e9, "cores": 1, "points_per_s": m1 / dt1,
                              "sample": f"{m1}-point subsample ({m1 * m1} pair tests, {dt1:.2f} s)"}}


def roofline(dom: str, avg_ms: float, ev: list, n: int, d: int, gs, wl_name: str, traffic, folded: bool = False):
    """Roofline of the dominant kernel from its CUDA-event time and the pairs it evaluated.

    Pair kernels: the tensor-core passes against the measured bf16 peak (2K FLOPs
    per pair, K = d padded to 16) with the epilogue's FP32 operations per pair
    beside it (about 3; 1.5 for the folded FP16 count, whose MMA also runs one
    more K chunk of 16: the MMA work it executes is reported beside the useful
    work); CUDA-core pair kernels (all-pairs tile and the eps-grid's count,
    merge and border) against the FP32 pipe at d+2 (Gram form) or 2d+1 (direct
    form) operations per evaluated pair, with the eps-grid kernels' HBM
    fraction beside it.  Other kernels against HBM."""
    peaks = load_peaks()
    sec = avg_ms * 1e-3
    if dom in PASS_OF:
        pairs = ev[PASS_OF[dom]]
        if dom.startswith("tc_"):
            K = -(-d // 16) * 16
            flops = 2.0 * pairs * K
            ach = flops / sec / 1e12
            roof = {"kernel": dom, "bound": "tensor", "achieved": ach, "peak": peaks["bf16_tflops"],
                    "unit": "TFLOP/s", "frac": ach / peaks["bf16_tflops"], "traffic": traffic,
                    "peak_src": peaks["src"] + " bf16 burst (FP16 dense rate is the same)",
                    "algorithmic_flops": flops, "pairs": pairs, "avg_ms": avg_ms}
            fp32_peak, _ = fp32_peak_tops()
            opp = 1.5 if (folded and dom == "tc_count") else 3
            alu = opp * pairs / sec / 1e12
            roof["epilogue_fp32"] = {"ops_per_pair": opp, "achieved": alu, "peak": fp32_peak, "unit": "T ops/s",
                                     "frac": alu / fp32_peak}
            if folded and dom == "tc_count":
                ex = 2.0 * pairs * (K + 16) / sec / 1e12
                roof["mma_executed"] = {"flops_per_pair": 2 * (K + 16), "achieved": ex, "unit": "TFLOP/s",
                                        "frac": ex / peaks["bf16_tflops"],
                                        "note": "the folded count's MMA runs K + 16 columns; frac above counts 2K"}
            return roof
        ops_pp = pair_ops(d) if not dom.startswith(("grid_", "mid_")) else d + 2
        fp32_peak, sms = fp32_peak_tops()
        ach = pairs * ops_pp / sec / 1e12
        alu = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "T FP32-pipe ops/s",
               "frac": ach / fp32_peak, "traffic": traffic, "peak_src": f"{sms} SMs x 128 lanes x max SM clock",
               "pairs": pairs, "ops_per_pair": ops_pp, "avg_ms": avg_ms}
        bound, work = algorithmic_work(dom, n, d, gs)
        if bound != "hbm" or not work:
            return alu
        # The eps-grid pair kernels move more bytes than they compute: the bound is
        # the larger of the two roofline times (FP32 ops / FP32 peak, bytes / HBM peak).
        gbs = work / sec / 1e9
        hbm = {"kernel": dom, "bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
               "frac": gbs / peaks["hbm_gbs"], "traffic": traffic if traffic is not None else ncu_traffic(wl_name, dom),
               "peak_src": peaks["src"], "algorithmic_bytes": work, "pairs": pairs, "avg_ms": avg_ms}
        t_alu = pairs * ops_pp / (fp32_peak * 1e12)
        t_hbm = work / (peaks["hbm_gbs"] * 1e9)
        main, other = (hbm, alu) if t_hbm >= t_alu else (alu, hbm)
        main["other_bound"] = {k: other[k] for k in ("bound", "achieved", "peak", "unit", "frac")}
        main["roofline_times_us"] = {"alu": t_alu * 1e6, "hbm": t_hbm * 1e6}
        return main
    bound, work = algorithmic_work(dom, n, d, gs)
    if bound == "hbm" and work:
        ach = work / sec / 1e9
        return {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": ach / peaks["hbm_gbs"], "traffic": traffic if traffic is not None else ncu_traffic(wl_name, dom),
                "peak_src": peaks["src"], "algorithmic_bytes": work, "avg_ms": avg_ms}
    return {"kernel": dom, "bound": bound, "achieved": None, "peak": None, "unit": None, "frac": None,
            "traffic": None, "avg_ms": avg_ms}


def run_ours(args, wl_name, baseline=True, steps=None):
    """Full record of one single-instance workload (dbscan_run on device buffers)."""
    from paper_1506_02226_gb300 import build as cuda_build
    cuda_build.build()  # in-tree, only recompiles what changed
    import torch
    from paper_1506_02226_gb300 import binding as B
    from paper_1506_02226_gb300.api import Plan

    steps = steps or args.steps
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as tdist
        if not tdist.is_initialized():
            tdist.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist = tdist

    desc, make = WORKLOADS[wl_name]
    inst = make()
    if args.n and args.n < inst.n:  # smaller sample of the same recipe (profiler captures)
        inst = inputs.subsample(inst, args.n, seed=0)
        desc = f"{args.n}-point uniform subsample of the {desc} workload"
    n, d = inst.n, inst.d
    x = torch.from_numpy(inst.points).cuda()
    labels = torch.empty(n, dtype=torch.int32, device="cuda")
    stream = torch.cuda.Stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    prec = PRECISION.get(wl_name, 0)
    # one synchronous run for the statistics (and the launch count)
    with Plan(max_n=n, max_d=d, precision=prec) as p:
        _, st0 = p.run(x, inst.eps, inst.min_pts, stats=True)
    candidates = st0["candidate_pairs"]
    gs = None
    if st0["path"] == B.DBSCAN_PATH_GRID:
        gs = grid_structure(inst.points, inst.eps)
        if gs["candidate_pairs"] != candidates:
            raise RuntimeError(f"candidate-pair count mismatch: device {candidates} host {gs['candidate_pairs']}")

    # Timed steps run without per-kernel marks, so the grid path's independent
    # kernels may overlap on its second stream; per-kernel times come from a
    # separate profiled plan that runs them one after another.
    plan = Plan(max_n=n, max_d=d, synchronous=False, stream=stream, profile=False, precision=prec)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    step_ms, step_pairs = [], []
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            plan.run(x, inst.eps, inst.min_pts, labels=labels)
        if plan.sync() != 0:
            raise RuntimeError("warm-up run reported an error")
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        clocks = ClockSampler(local)
        time.sleep(0.3)
        for _ in range(steps):
            flush.fill_(1)  # evict the 129 MB L2 before the timed step
            ev0.record(stream)
            plan.run(x, inst.eps, inst.min_pts, labels=labels)
            ev1.record(stream)
            ev1.synchronize()
            step_ms.append(ev0.elapsed_time(ev1))
            step_pairs.append(sum(plan.pair_tests()))  # this step's device counters (outside the events)
        torch.cuda.synchronize()
        clk = clocks.stop()
    if plan.sync() != 0:
        raise RuntimeError("timed run reported an error")
    kern: dict[str, list[float]] = {}
    ev_runs = []
    pplan = Plan(max_n=n, max_d=d, synchronous=False, stream=stream, profile=True, precision=prec)
    with torch.cuda.stream(stream):
        for r in range(3 + max(5, min(steps, 30))):
            flush.fill_(1)
            pplan.run(x, inst.eps, inst.min_pts, labels=labels)
            stream.synchronize()
            if r >= 3:
                for nm, ms in pplan.phase_times():
                    kern.setdefault(nm, []).append(ms)
                ev_runs.append(pplan.pair_tests())
    if pplan.sync() != 0:
        raise RuntimeError("profiled run reported an error")
    # FP16 tensor-core count: whether it ran the folded form (counter slot 15)
    tc_form = None
    if st0["path"] == B.DBSCAN_PATH_ALLPAIRS_TC and prec != B.DBSCAN_PREC_BF16_GRAM:
        tc_form = "folded (column norm inside the MMA)" if pplan.counters()[15] else "G alone"
    pplan.close()
    total_ms = max_over_ranks(sum(step_ms), dist, "cuda")
    if dist:
        dist.barrier()
    ms_per_step = total_ms / steps
    pairs_per_step = statistics.mean(step_pairs)
    value = whole_job_rate(pairs_per_step, world, ms_per_step) / 1e9

    # end to end: host (pinned) buffers through the C ABI, copies inside the timed region
    host_pts = torch.from_numpy(inst.points).pin_memory()
    host_lab = torch.empty(n, dtype=torch.int32).pin_memory()
    eplan = Plan(max_n=n, max_d=d, stream=stream, precision=prec)
    for _ in range(2):
        eplan.run_host(host_pts, inst.eps, inst.min_pts, labels=host_lab)
    e2e_s = []
    for _ in range(max(3, steps // 4) if not args.no_baseline else 1):
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        eplan.run_host(host_pts, inst.eps, inst.min_pts, labels=host_lab)
        e2e_s.append(time.perf_counter() - t0)
    e2e_ms = 1e3 * statistics.mean(e2e_s)
    eplan.close()
    plan.close()
    allpairs = None
    if wl_name in COMPARE_ALLPAIRS:  # the same instance with the grid off (the paper's all-pairs test)
        aplan = Plan(max_n=n, max_d=d, synchronous=False, stream=stream, grid=B.DBSCAN_GRID_OFF, precision=prec)
        a_ms = []
        with torch.cuda.stream(stream):
            for r in range(2 + 3):
                flush.fill_(1)
                ev0.record(stream)
                aplan.run(x, inst.eps, inst.min_pts, labels=labels)
                ev1.record(stream)
                ev1.synchronize()
                if r >= 2:
                    a_ms.append(ev0.elapsed_time(ev1))
        if aplan.sync() != 0:
            raise RuntimeError("all-pairs comparison run reported an error")
        a_pairs = sum(aplan.pair_tests())
        aplan.close()
        allpairs = {"ms_per_step": statistics.mean(a_ms), "pair_tests_per_step": a_pairs,
                    "speedup_of_grid": statistics.mean(a_ms) / ms_per_step,
                    "what": "the same instance on the all-pairs CUDA-core path (grid off), 3 steps"}

    if rank != 0:
        return None
    avg = {k: statistics.mean(v) for k, v in kern.items()}
    ev_pass = [statistics.mean(r[k] for r in ev_runs) for k in range(4)]
    dom = max(avg, key=avg.get)
    folded = tc_form is not None and tc_form.startswith("folded")
    roof = roofline(dom, avg[dom], ev_pass, n, d, gs, wl_name, args.traffic, folded)
    others = {}
    for k in sorted(avg, key=avg.get, reverse=True)[1:4]:
        if k in PASS_OF and ev_pass[PASS_OF[k]] > 0:
            r = roofline(k, avg[k], ev_pass, n, d, gs, wl_name, None, folded)
            others[k] = {"bound": r["bound"], "frac": r["frac"], "achieved": r["achieved"], "unit": r["unit"],
                         "pairs": r.get("pairs"), "avg_ms": avg[k]}
    cpu = cpu_baseline(inst, wl_name, desc) if (baseline and not args.no_baseline) else None
    return {
        "metric": "G pair-tests/s", "value": value, "unit": "G pair-tests/s", "n_gpus": world,
        "steps": steps, "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": {2: "f32", 3: "f16" if prec != 3 else "bf16"}.get(
            st0["path"], "f32"), "data": "synthetic",
        "config": {"workload": wl_name + ": " + desc, "n": n, "d": d, "eps": inst.eps, "min_pts": inst.min_pts,
                   "path": {1: "eps-grid", 2: "all-pairs SIMT", 3: "all-pairs tensor-core",
                            4: "projected grid"}.get(st0["path"]),
                   "l2": "flushed by a 256 MiB write before every timed step", "parallelism": f"replicas x{world}"},
        "pair_tests_per_step": pairs_per_step,
        "pair_tests_by_pass": dict(zip(["count", "merge", "border", "merge_outer_ring"], ev_pass)),
        "pair_tests_note": "pair predicates the device evaluated (its per-pass counters), averaged over the "
                           "timed steps; pairs decided without a test are not counted",
        "candidate_pairs_per_step": (candidates if st0["path"] in (B.DBSCAN_PATH_GRID, B.DBSCAN_PATH_GRID_PROJECTED)
                                     else n * n),
        "evaluated_vs_min": pairs_per_step / max(n * (n - 1) / 2, 1),
        "band_pairs_per_step": st0["band_pairs"],
        "tc_count_form": tc_form,
        "points_per_s": world * n / (ms_per_step * 1e-3),
        "clusters": st0["n_clusters"], "core": st0["n_core"], "noise": st0["n_noise"],
        "kernels_ms": {k: round(v, 5) for k, v in sorted(avg.items(), key=lambda kv: -kv[1])},
        "kernels_ms_note": "each kernel alone (a profiled run, kernels serialised, L2 flushed before each run)",
        "roofline": roof,
        "roofline_next": others,
        "allpairs": allpairs,
        "cpu_baseline": cpu,
        "e2e": {"value": pairs_per_step / (e2e_ms * 1e-3) / 1e9, "unit": "G pair-tests/s", "ms_per_step": e2e_ms,
                "points_per_s": n / (e2e_ms * 1e-3), "h2d_bytes_per_step": 4 * n * d, "d2h_bytes_per_step": 4 * n},
        "gpu_launches": st0["kernels"] * steps,
        "clocks": clk,
    }


def run_batch(args, steps=None):
    """4,096 independent instances per step, one dbscan_batch call (graph launch)."""
    steps = steps or args.steps
    from paper_1506_02226_gb300 import build as cuda_build
    cuda_build.build()
    import torch
    from paper_1506_02226_gb300 import binding as B
    from paper_1506_02226_gb300.api import Plan

    insts = inputs.batch(count=args.batch_count)
    count = len(insts)
    sizes = [i.n * i.d for i in insts]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    loffs = np.concatenate([[0], np.cumsum([i.n for i in insts])])
    host_pts = torch.from_numpy(np.concatenate([i.points.reshape(-1) for i in insts])).pin_memory()
    x = host_pts.cuda()
    lab = torch.empty(int(loffs[-1]), dtype=torch.int32, device="cuda")
    host_lab = torch.empty(int(loffs[-1]), dtype=torch.int32).pin_memory()

    def table(xbase, lbase):
        arr = (B.dbscan_instance * count)()
        for k, inst in enumerate(insts):
            arr[k].points = xbase + 4 * int(offs[k])
            arr[k].n = inst.n
            arr[k].d = inst.d
            arr[k].eps = inst.eps
            arr[k].min_pts = inst.min_pts
            arr[k].labels_out = lbase + 4 * int(loffs[k])
        return arr

    arr = table(x.data_ptr(), lab.data_ptr())
    stream = torch.cuda.Stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    plan = Plan(max_n=16, max_d=16, stream=stream)
    st = (B.dbscan_stats * count)()
    if B.dbscan_batch(plan.handle, arr, st) != 0:  # autotune + graph capture
        raise RuntimeError("dbscan_batch failed")
    ch, bps = B.dbscan_batch_config(plan.handle)
    tile_rows, tile_cols = B.dbscan_batch_tile(plan.handle)
    ncore = [st[k].n_core for k in range(count)]
    pair_tests = sum(st[k].pair_tests for k in range(count))  # device counters of that call
    pass_pairs = B.dbscan_plan_counters(plan.handle)[16:19]  # that call's totals per pass
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            B.dbscan_batch(plan.handle, arr)
        clocks = ClockSampler(torch.cuda.current_device())
        time.sleep(0.3)
        step_ms = []
        for _ in range(steps):
            flush.fill_(1)
            ev0.record(stream)
            if B.dbscan_batch(plan.handle, arr) != 0:
                raise RuntimeError("dbscan_batch failed")
            ev1.record(stream)
            ev1.synchronize()
            step_ms.append(ev0.elapsed_time(ev1))
        clk = clocks.stop()
        # per-kernel times: one profiled (uncaptured) run
        pplan = Plan(max_n=16, max_d=16, stream=stream, profile=True)
        B.dbscan_batch(pplan.handle, arr)
        B.dbscan_batch(pplan.handle, arr)
        kern = dict(pplan.phase_times())
        pplan.close()
        # the same instances through a loop of single-instance launches
        single = Plan(max_n=8192, max_d=16, stream=stream, synchronous=False)
        loop_ms = []
        for _ in range(max(2, steps // 10)):
            flush.fill_(1)
            ev0.record(stream)
            for k, inst in enumerate(insts):
                B.dbscan_run(single.handle, arr[k].points, inst.n, inst.d, inst.eps, inst.min_pts, arr[k].labels_out)
            ev1.record(stream)
            ev1.synchronize()
            loop_ms.append(ev0.elapsed_time(ev1))
        if single.sync() != 0:
            raise RuntimeError("single-instance loop failed")
        single.close()
        # end to end: host buffers in, labels out, every step
        harr = table(x.data_ptr(), lab.data_ptr())
        e2e = []
        for _ in range(max(3, steps // 4)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            x.copy_(host_pts, non_blocking=True)
            B.dbscan_batch(plan.handle, harr)
            host_lab.copy_(lab, non_blocking=True)
            torch.cuda.synchronize()
            e2e.append(time.perf_counter() - t0)
    plan.close()
    ms = statistics.mean(step_ms)
    jobs = count / (ms * 1e-3)
    pairs = sum(i.n * i.n for i in insts)
    peak_tops, sms = fp32_peak_tops()
    dom = max(kern, key=kern.get)
    if dom in ("batch_count", "batch_union", "batch_border"):
        # pairs each pass evaluated (device counters of a batch run with statistics)
        # times the FP32-pipe operations of one pair test at the instance's d
        k = ("batch_count", "batch_union", "batch_border").index(dom)
        pp = pass_pairs[k]
        mean_ops = sum(i.n * i.n * pair_ops(i.d) for i in insts) / max(sum(i.n * i.n for i in insts), 1)
        ops = pp * mean_ops
        ach = ops / (kern[dom] * 1e-3) / 1e12
        roof = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": peak_tops, "unit": "T FP32-pipe ops/s",
                "frac": ach / peak_tops, "traffic": args.traffic, "peak_src": f"{sms} SMs x 128 lanes x max clock",
                "avg_ms": kern[dom]}
    else:
        roof = {"kernel": dom, "bound": None, "achieved": None, "peak": None, "unit": None, "frac": None,
                "traffic": None, "avg_ms": kern[dom]}
    cpu = None
    if not args.no_baseline:
        import oracle
        sample = insts[:args.cpu_sample]
        cores = os.cpu_count() or 1
        t0 = time.perf_counter()
        for inst in sample:
            oracle.dbscan(inst.points, inst.eps, inst.min_pts, nthreads=cores)
        dt = time.perf_counter() - t0
        cpu = {"value": len(sample) / dt, "unit": "jobs/s", "cores": cores, "kind": "oracle",
               "sample": f"the first {len(sample)} of the {count} instances, run one after another ({dt:.2f} s)"}
    e2e_ms = 1e3 * statistics.mean(e2e)
    out = {
        "metric": "batched jobs/s", "value": jobs, "unit": "jobs/s", "n_gpus": 1, "steps": steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"batch: {count} instances, n log-uniform 64..8192, d in {{2,3,16}}, 1-8 blobs + 10% "
                               "noise, eps U[0.01,0.05], min_pts U{4..16}", "points": int(loffs[-1]),
                   "path": "all-pairs SIMT, one graph launch",
                   "autotuned": {"tile": [tile_rows, tile_cols], "chunk_tiles": ch, "blocks_per_sm": bps},
                   "l2": "flushed by a 256 MiB write before every timed step"},
        "pair_tests_per_step": pair_tests, "pair_tests_per_s": pair_tests / (ms * 1e-3),
        "pair_tests_by_pass": {"count": int(pass_pairs[0]), "merge": int(pass_pairs[1]), "border": int(pass_pairs[2])},
        "all_pairs_per_step": pairs,
        "launch_loop": {"jobs_per_s": count / (statistics.mean(loop_ms) * 1e-3), "ms": statistics.mean(loop_ms),
                        "what": "the same instances, one dbscan_run per instance on one stream"},
        "kernels_ms": {k: round(v, 5) for k, v in sorted(kern.items(), key=lambda kv: -kv[1])},
        "roofline": roof, "cpu_baseline": cpu,
        "e2e": {"value": count / (e2e_ms * 1e-3), "unit": "jobs/s", "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": 4 * int(offs[-1]), "d2h_bytes_per_step": 4 * int(loffs[-1])},
        "gpu_launches": 6 * steps, "clocks": clk,
    }
    return out


def run_serve(args):
    """Jobs through the server: closed-loop saturation, then Poisson arrivals at
    0.7x and 0.9x of it, with per-job submit-to-done latency; beside it the same
    jobs through a plain loop of dbscan_run calls on one stream."""
    from paper_1506_02226_gb300 import build as cuda_build
    cuda_build.build()
    import threading
    import torch
    from paper_1506_02226_gb300 import binding as B
    from paper_1506_02226_gb300.api import Plan

    pool = [inputs.serve_job(i) for i in range(args.serve_pool)]
    dev = []
    for inst in pool:
        x = torch.from_numpy(inst.points).cuda()
        lab = torch.empty(inst.n, dtype=torch.int32, device="cuda")
        s = B.dbscan_instance()
        s.points, s.n, s.d, s.eps, s.min_pts, s.labels_out = x.data_ptr(), inst.n, inst.d, inst.eps, inst.min_pts, \
            lab.data_ptr()
        dev.append((x, lab, s))
    max_n = max(i.n for i in pool)
    njobs = args.serve_jobs

    # the plain loop: one plan sized for the largest job, one stream, one
    # dbscan_run per job in submission order, waited for at the end
    stream = torch.cuda.Stream()
    loop_jobs = min(njobs, args.serve_loop_jobs)
    with Plan(max_n=max_n, max_d=64, synchronous=False, stream=stream) as single:
        for k in range(min(len(dev), 16)):  # warm-up (first launches of every kernel)
            s = dev[k][2]
            B.dbscan_run(single.handle, s.points, s.n, s.d, s.eps, s.min_pts, s.labels_out)
        if single.sync() != 0:
            raise RuntimeError("launch loop warm-up failed")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(loop_jobs):
            s = dev[k % len(dev)][2]
            B.dbscan_run(single.handle, s.points, s.n, s.d, s.eps, s.min_pts, s.labels_out)
        if single.sync() != 0:
            raise RuntimeError("launch loop failed")
        loop_s = time.perf_counter() - t0

    o = B.dbscan_serve_opts_default()
    o.slots = args.serve_slots
    o.max_n = max_n
    o.max_d = 64
    srv = B.dbscan_serve_create(o)

    def run(arrivals):
        ids, lats = [None] * njobs, [0.0] * njobs
        t0 = time.perf_counter()

        def submitter():
            for k in range(njobs):
                if arrivals is not None:
                    dt = arrivals[k] - (time.perf_counter() - t0)
                    if dt > 0:
                        time.sleep(dt)
                ids[k] = B.dbscan_serve_submit(srv, dev[k % len(dev)][2])

        th = threading.Thread(target=submitter)
        th.start()
        for k in range(njobs):
            while ids[k] is None:
                time.sleep(50e-6)
            st, lat = B.dbscan_serve_wait(srv, ids[k], -1)
            if st != 0:
                raise RuntimeError(f"serve job {k} failed: {st}")
            lats[k] = lat
        th.join()
        wall = time.perf_counter() - t0
        return njobs / wall, lats

    for k in range(min(len(dev), 2 * args.serve_slots)):  # warm-up: first launches, graph/attribute setup
        B.dbscan_serve_wait(srv, B.dbscan_serve_submit(srv, dev[k][2]), -1)
    clocks = ClockSampler(torch.cuda.current_device())
    sat, lat_closed = run(None)
    levels = {}
    for frac in (0.7, 0.9):
        arr = inputs.serve_arrivals(njobs, frac * sat)
        jobs_s, lats = run(arr)
        levels[str(frac)] = {"offered_jobs_per_s": frac * sat, "jobs_per_s": jobs_s,
                             "p50_ms": float(np.percentile(lats, 50)) / 1e3,
                             "p99_ms": float(np.percentile(lats, 99)) / 1e3}
    clk = clocks.stop()
    info = B.dbscan_serve_info(srv) if hasattr(B, "dbscan_serve_info") else None
    B.dbscan_serve_destroy(srv)
    mix = {d: sum(1 for i in pool if i.d == d) for d in (2, 3, 32)}
    return {
        "metric": "served jobs/s", "value": sat, "unit": "jobs/s", "n_gpus": 1, "steps": njobs, "warmup":
            min(len(dev), 2 * args.serve_slots), "ms_per_step": 1e3 / sat, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"serve: {njobs} jobs drawn cyclically from {len(pool)} seeded jobs, n log-uniform "
                               f"1k..500k, d in {{2,3,32}} ({mix}), blob+noise, per-job eps/min_pts",
                   "slots": args.serve_slots, "hbm_budget_gib": o.hbm_budget_bytes / 2 ** 30},
        "closed_loop": {"jobs_per_s": sat, "p50_ms": float(np.percentile(lat_closed, 50)) / 1e3,
                        "p99_ms": float(np.percentile(lat_closed, 99)) / 1e3,
                        "note": "all jobs submitted at once: latency includes queueing behind the whole stream"},
        "poisson": levels,
        "launch_loop": {"jobs_per_s": loop_jobs / loop_s, "jobs": loop_jobs,
                        "what": "the first jobs of the same stream, one dbscan_run per job on one stream and one "
                                "plan sized for the largest job"},
        "server_memory": info,
        "e2e": None, "roofline": None, "cpu_baseline": None, "gpu_launches": None, "clocks": clk,
    }


def run_paper_compare(args, n=23_040, steps=3):
    """The paper's materialised pipeline (dbscan_run_paper: distance matrix,
    primitive-cluster matrix, one merge launch per target) against this
    library's fused all-pairs and eps-grid runs on the same 3-D input."""
    from paper_1506_02226_gb300 import build as cuda_build
    cuda_build.build()
    import torch
    from paper_1506_02226_gb300 import binding as B
    from paper_1506_02226_gb300.api import Plan
    inst = inputs.paper_3d(n)
    x = torch.from_numpy(inst.points).cuda()
    lab = torch.empty(n, dtype=torch.int32, device="cuda")
    out = {"workload": f"paper3d: {n} points, d=3, 50 blobs + 20% noise, eps=0.02, min_pts=10 (synthetic stand-in "
                       "for the paper's unnamed 3-D set at its N)", "n": n}
    with Plan(max_n=n, max_d=3, profile=True) as p:
        phases, total = {}, []
        for r in range(1 + steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, st = p.run_paper(x, inst.eps, inst.min_pts, labels=lab, stats=True)
            wall = time.perf_counter() - t0
            if r >= 1:
                total.append(wall * 1e3)
                for nm, ms in p.phase_times():
                    phases.setdefault(nm, []).append(ms)
        want = lab.cpu().numpy().copy()
        out["paper_pipeline"] = {"ms_per_run": statistics.mean(total), "merge_sweeps": st["cells"],
                                 "phases_ms": {k: statistics.mean(v) for k, v in phases.items()},
                                 "what": "Section IV as the paper builds it: N x N distance matrix, primitive-cluster "
                                         "matrix and valid vector, one merge launch per valid target per sweep "
                                         "(host-driven, wall clock)"}
    for name, grid in (("fused_allpairs", B.DBSCAN_GRID_OFF), ("grid", B.DBSCAN_GRID_AUTO)):
        with Plan(max_n=n, max_d=3, grid=grid, profile=True) as p:
            ts = []
            for r in range(3 + steps):
                _, st = p.run(x, inst.eps, inst.min_pts, labels=lab, stats=True)
                if r >= 3:
                    ts.append(st["ms_total"])
            got = lab.cpu().numpy()
            if not np.array_equal(got, want):
                raise RuntimeError(f"paper pipeline and {name} labels differ")
            out[name] = {"ms_per_run": statistics.mean(ts), "phases_ms": dict(p.phase_times())}
    out["speedup_fused_over_paper"] = out["paper_pipeline"]["ms_per_run"] / out["fused_allpairs"]["ms_per_run"]
    out["speedup_grid_over_paper"] = out["paper_pipeline"]["ms_per_run"] / out["grid"]["ms_per_run"]
    out["labels_identical"] = True
    return out


def compact(rec: dict) -> dict:
    """The figures of a workload's record that the default line carries."""
    keep = ("metric", "value", "unit", "ms_per_step", "dtype", "pair_tests_per_step", "candidate_pairs_per_step",
            "evaluated_vs_min", "band_pairs_per_step", "tc_count_form", "points_per_s", "launch_loop", "closed_loop",
            "poisson",
            "server_memory", "allpairs", "config", "clocks")
    out = {k: rec[k] for k in keep if k in rec}
    r = rec.get("roofline")
    if r:
        out["roofline"] = {k: r[k] for k in ("kernel", "bound", "achieved", "peak", "unit", "frac", "avg_ms",
                                             "epilogue_fp32", "mma_executed", "other_bound") if k in r}
    if rec.get("e2e"):
        out["e2e"] = {k: rec["e2e"][k] for k in ("value", "unit", "ms_per_step") if k in rec["e2e"]}
    if rec.get("cpu_baseline"):
        out["cpu_baseline"] = {k: rec["cpu_baseline"][k] for k in ("value", "unit", "cores", "sample")}
    if "kernels_ms" in rec:
        out["kernels_ms"] = dict(list(rec["kernels_ms"].items())[:4])
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["batch", "serve", "paper"], default=None,
                    help="print the full record of one workload (default: lowd2 with the others as subrecords)")
    ap.add_argument("--no-subrecords", action="store_true", help="default run without the other workloads")
    ap.add_argument("--no-baseline", action="store_true", help="skip the CPU baseline (for profiler runs)")
    ap.add_argument("--n", type=int, default=0, help="cluster a uniform subsample of this many points instead")
    ap.add_argument("--batch-count", type=int, default=4096, help="instances of the batch workload")
    ap.add_argument("--serve-jobs", type=int, default=10_000, help="jobs of the serve workload")
    ap.add_argument("--serve-pool", type=int, default=192, help="distinct seeded jobs the serve workload cycles")
    ap.add_argument("--serve-slots", type=int, default=8, help="server slots")
    ap.add_argument("--serve-loop-jobs", type=int, default=2000, help="jobs of the plain launch loop beside serve")
    ap.add_argument("--cpu-sample", type=int, default=128, help="instances the oracle runs for the batch baseline")
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per launch of the dominant kernel from an ncu capture, for the roofline")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    wl = args.workload
    if args.impl == "reference":
        if int(os.environ.get("RANK", "0")) != 0:
            return
        run_reference(args, wl or "lowd2")
        return
    if wl == "batch":
        print(json.dumps(run_batch(args)))
        return
    if wl == "serve":
        print(json.dumps(run_serve(args)))
        return
    if wl == "paper":
        print(json.dumps(run_paper_compare(args)))
        return
    if wl is not None:
        rec = run_ours(args, wl)
        if rec is not None:
            print(json.dumps(rec))
        return
    rec = run_ours(args, "lowd2")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rec is not None and world == 1 and not args.no_subrecords:
        sub = {}
        sub["lowd3"] = compact(run_ours(args, "lowd3", baseline=False))
        sub["highd_fp16"] = compact(run_ours(args, "highd", steps=min(args.steps, 10)))
        sub["highd_bf16"] = compact(run_ours(args, "highd_bf16", baseline=False, steps=min(args.steps, 10)))
        sub["midd8"] = compact(run_ours(args, "midd8", baseline=False, steps=min(args.steps, 10)))
        sub["batch"] = compact(run_batch(args, steps=min(args.steps, 10)))
        sub["serve"] = compact(run_serve(args))
        sub["paper_pipeline"] = run_paper_compare(args)
        rec["subrecords"] = sub
    if rec is not None:
        print(json.dumps(rec))
    if world > 1:
        import torch.distributed as tdist
        if tdist.is_initialized():
            tdist.destroy_process_group()


if __name__ == "__main__":
    main()
