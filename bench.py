#!/usr/bin/env python
"""Benchmark: filtered exact top-k queries/s on the 1M x 128 fp32 workload.

Workload (one cell of the 1M-row sweep; synthetic, seeded): 1,000,000 rows,
d = 128 float32 from a 64-centre Gaussian mixture (centre std 1, within std
0.3); one int32 attribute uniform on [0, 10^6); predicate attr < s * 10^6;
a batch of B queries from the same mixture; k = 10; squared L2.  Defaults:
B = 16, s = 10%.  One step = one batch through the whole path (predicate,
compaction, distance pass with fused top-k', merge, exact re-rank).

Timing: W warm-up steps, then K timed steps.  Before every step the L2 cache
is flushed by writing a 256 MiB buffer and then reading another one, so the
timed step starts with no useful and no dirty lines in L2 (the flush is
outside the timed interval); each
step is bracketed by CUDA events on the query's stream and the value is
B * K / (sum of step times).  The library's own stage events (same stream)
give the distance kernel's average duration for the roofline.  e2e repeats
the measurement through the C ABI with pinned host buffers (query upload
and result download inside the timed interval, host-clock timed).

--impl reference times the CPU oracle (float64, full sort) on the same
workload; it is the baseline arm, not the optimisation target.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import gen  # noqa: E402

FALLBACK_HBM_GBS = 6800.0
FLUSH_BYTES = 256 << 20
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")
# the dense-key distance pass of the float32 GEMV plan at 1-64 queries runs
# on the tensor cores by default (VRS_OPT_TENSOR_GEMV)
DIST_KERNEL = "umma_pair_kernel"
# what each kernel compiles: its file, the PTX wrappers, and from the shared
# header only its argument struct ("file:Struct")
KERNEL_SOURCES = {
    "scan_simt_kernel": ["k_scan_simt.cu", "topk_select.cuh", "vrs_internal.cuh:ScanArgs"],
    "umma_rows_kernel": ["k_umma_rows.cu", "umma.cuh", "vrs_internal.cuh:ScanArgs"],
    "umma_pair_kernel": ["k_umma_pair.cu", "umma.cuh", "vrs_internal.cuh:ScanArgs"],
}
# selectivities of the default sweep (the metric's axis), at the headline batch
SEL_AXIS = (0.001, 0.01, 0.1, 0.5, 1.0)


def parse():
    p = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["vrs", "reference"], default="vrs")
    p.add_argument("--workload", choices=["sweep", "precision", "batched", "learned", "peaks",
                                          "range", "join", "dnf"],
                   default="sweep",
                   help="sweep: 1M x 128 fp32 cell (default); precision: 1M x 960 with "
                        "bf16/e4m3 copies; batched: 10M x 96 bf16, per-query predicates; "
                        "range / join / dnf: range search, vector join and disjunctions "
                        "on the 1M x 128 table")
    p.add_argument("--compute", choices=["f32", "bf16", "fp8"], default="bf16",
                   help="first-pass arithmetic of the precision workload")
    p.add_argument("--no-pair-copy", action="store_true",
                   help="sweep workload: the float32 rows' 3xTF32 GEMV pass (umma_rows_kernel) "
                        "instead of the bf16 pair copy's (umma_pair_kernel)")
    p.add_argument("--no-grid", action="store_true",
                   help="batched workload: no grid index (the mask plan runs)")
    p.add_argument("--no-bf16-copy", action="store_true",
                   help="precision workload: load no bf16 copy, so E4M3 requests run on E4M3")
    p.add_argument("--n", type=int, default=None)
    p.add_argument("--d", type=int, default=None)
    p.add_argument("--batch", type=int, default=None)
    p.add_argument("--sel", type=float, default=0.10)
    p.add_argument("--k", type=int, default=10)
    p.add_argument("--metric", choices=["l2", "ip"], default="l2")
    p.add_argument("--sweep", action="store_true",
                   help="also time the whole B x s grid (1, 16, 256, 1024 queries)")
    p.add_argument("--no-sel-sweep", action="store_true",
                   help="skip the default selectivity sweep at the headline batch")
    p.add_argument("--shard", choices=["none", "rows"], default="none",
                   help="rows: each rank holds a contiguous row range of the table and "
                        "answers the same query batch; the ranks all-gather their top-k "
                        "lists and merge them (strong scaling)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=10.0)
    return p.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload(args):
    wl = gen.sweep_cell(args.batch or 16, args.sel, args.k, args.metric, n=args.n or 1_000_000,
                        d=args.d or 128)
    return wl


def load_inputs(wl, rank: int):
    """Rows, attributes and this rank's query batch (rank r takes the r-th
    batch of B queries drawn from the mixture's query stream)."""
    mix = wl.mixture()
    x = gen.vectors(wl.n, mix, unit=wl.unit)
    attrs = gen.attributes(wl.n, 1, wl.attr_range)
    q = gen.queries(wl.batch * (rank + 1), mix, unit=wl.unit)[rank * wl.batch:]
    return x, attrs, np.ascontiguousarray(q)


def config_of(wl, args):
    return {
        "workload": wl.name,
        "n": wl.n, "d": wl.d, "batch": wl.batch, "selectivity": wl.selectivity,
        "k": wl.k, "metric": wl.metric, "storage": "f32",
        "data": "gaussian mixture, 64 centres, seed 0",
        "l2": "flushed before every step (256 MiB write, then 256 MiB read)",
    }


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def kernel_hash(name):
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[name]:
        f, _, struct = f.partition(":")
        with open(os.path.join(ROOT, "paper_2403_15807_gb300", "csrc", f), "rb") as fh:
            src = fh.read()
        if struct:
            i = src.index(b"struct " + struct.encode() + b" {")
            src = src[i:src.index(b"};", i)]
        h.update(src)
    return h.hexdigest()[:16]


def recorded_traffic(name, cell):
    """DRAM bytes per launch from a committed ncu capture, if the kernel's
    sources are unchanged since it was taken."""
    try:
        with open(TRAFFIC_FILE) as f:
            t = json.load(f)
        e = t[name]
        if e.get("source_hash") != kernel_hash(name) or e.get("cell") != cell:
            return None
        return float(e["dram_bytes_per_launch"])
    except Exception:
        return None


class Clocks:
    """nvidia-smi sampler running during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"vrs_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc:
            return None
        rows = []
        with open(self.path) as f:
            for line in f:
                p = [c.strip() for c in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    rows.append((float(p[1]), float(p[2]), p[5], p[6], p[7], p[8]))
                except ValueError:
                    continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[2 + i] == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def run_reference(args):
    """The CPU oracle on the same workload (float64, full sort, all cores)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    wl = workload(args)
    x, attrs, q = load_inputs(wl, 0)
    cores = os.cpu_count() or 1
    # each step: a bounded sample of the batch (the first min(B, cores) queries)
    qs = q[: max(1, min(wl.batch, cores))]
    pred = wl.pred()
    for _ in range(args.warmup):
        oracle.query(x, attrs, qs, [pred], wl.k, wl.metric, n_threads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.query(x, attrs, qs, [pred], wl.k, wl.metric, n_threads=cores)
    el = time.perf_counter() - t0
    qps = qs.shape[0] * args.steps / el
    sample = f"{qs.shape[0]} of the {wl.batch} queries per step, full {wl.n}-row table"
    line = {
        "impl": "reference", "metric": "filtered exact top-k queries/s (recall@k=1.0)",
        "value": qps, "unit": "queries/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_of(wl, args),
        "cpu_baseline": {"value": qps, "unit": "queries/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": qps, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline(wl, x, attrs, q, seconds):
    import oracle
    cores = os.cpu_count() or 1
    pred = wl.pred()
    qs = q[: max(1, min(wl.batch, cores))]
    t0 = time.perf_counter()
    done = 0
    while True:
        oracle.query(x, attrs, qs, [pred], wl.k, wl.metric, n_threads=cores)
        done += qs.shape[0]
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return {"value": done / el, "unit": "queries/s", "cores": cores, "kind": "oracle",
            "sample": f"batches of {qs.shape[0]} queries over the full {wl.n}-row table, "
                      f"repeated for {el:.1f} s"}


class L2Flush:
    """Evict L2: write one 256 MiB buffer, then read another (the read pass
    writes back the dirty lines outside the timed interval)."""

    def __init__(self, torch, dev):
        self.w = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        self.r = torch.ones(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        self.acc = torch.empty((), dtype=torch.float32, device=dev)

    def zero_(self):
        self.w.zero_()
        self.acc.copy_(self.r.sum())


def time_steps(torch, vrs, eng, qd, pred, k, metric, steps, warmup, flush, stream,
               compute=0, preds=None, ks=None):
    """Per-step CUDA-event times (ms) of `steps` queries submitted back to
    back (each after an L2 flush on the same stream, profiling off, so the
    host runs ahead of the device), then the per-stage times (ms) of a few
    more steps with the library's stage events on.  Returns (step times,
    distance-stage times, launches per timed step x steps, summed stage
    times scaled to `steps`, outputs)."""
    kk = np.int32([k]) if ks is None else ks
    k_max = int(kk.max())
    # predicates are marshalled into the C layout once, as a caller that
    # keeps them would (the binding otherwise packs them on every call)
    preds = vrs.PredArray([pred] if preds is None else preds)
    oid = torch.empty((qd.shape[0], k_max), dtype=torch.int64, device=qd.device)
    odist = torch.empty((qd.shape[0], k_max), dtype=torch.float32, device=qd.device)

    def one():
        vrs.vrs_query(eng.h, qd, preds, kk, k_max=k_max, metric=metric, compute=compute,
                      out_ids=oid, out_dist=odist, stream=stream)

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    vrs.vrs_set_option(eng.h, vrs.VRS_OPT_PROFILE, 0)
    with torch.cuda.stream(stream):
        for i in range(warmup + steps):
            flush.zero_()
            j = i - warmup
            if j >= 0:
                ev[j][0].record(stream)
            one()
            if j >= 0:
                ev[j][1].record(stream)
    torch.cuda.synchronize()
    times = [a.elapsed_time(b) for a, b in ev]
    # stage breakdown (the stage events sit between the kernels)
    vrs.vrs_set_option(eng.h, vrs.VRS_OPT_PROFILE, 1)
    n_prof = max(3, min(steps, 10))
    dist_ms, launches, stage_sum = [], 0, None
    with torch.cuda.stream(stream):
        for i in range(2 + n_prof):
            flush.zero_()
            one()
            st, nl, _ = vrs.vrs_last_profile(eng.h)
            if i >= 2:
                dist_ms.append(st["distance"])
                launches += nl
                stage_sum = st if stage_sum is None else {a: stage_sum[a] + st[a] for a in st}
    torch.cuda.synchronize()
    scale = steps / n_prof
    stage_sum = {a: v * scale for a, v in stage_sum.items()}
    return times, dist_ms, int(round(launches * scale)), stage_sum, (oid, odist)


def tensor_peak(compute):
    """Dense peak for the contraction's dtype: measured BF16 (sustained, the
    kernel runs inside a long step), E4M3 = 2x BF16 (nominal 4.5 / 2.25)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        bf = float(pk["bf16_tflops_sustained"])
        src = "measured (bf16 sustained)"
    except Exception:
        bf, src = 1700.0, "fallback (bf16 sustained)"
    if compute == 2:
        return 2.0 * bf, src + " x 2 for E4M3 (nominal ratio)"
    return bf, src


def run_learned(args):
    """Learned plan choice at N = 5e7, d = 128 bf16: the network is trained
    by the library's kernels on the engine's timing grid (plus the 5e7-row
    cells at other batch sizes) and scored on held-out 5e7-row cells against
    the fixed rule and the per-cell best plan, using the per-plan latencies
    the engine measured (paper_2403_15807_gb300/data)."""
    from paper_2403_15807_gb300 import planner, vrs
    vrs.load()
    data = os.path.join(ROOT, "paper_2403_15807_gb300", "data")
    grid = json.load(open(os.path.join(data, "timings_grid_gb300.json")))["records"]
    table = json.load(open(os.path.join(data, "timings_eval_gb300.json")))["records"]
    train, test = planner.split_50m(grid, table)
    t0 = time.perf_counter()
    m = planner.fit(train, steps=3000)
    train_s = time.perf_counter() - t0
    ev = planner.evaluate(m, test)
    nq = sum(r["b"] for r in test if all(r["ms"].get(p) is not None
                                         for p, ok in zip(planner.PLANS, planner.AVAILABLE["bf16"])
                                         if ok))
    line = {
        "metric": "filtered exact top-k queries/s (recall@k=1.0)",
        "value": nq / (ev["model"] / 1e3), "unit": "queries/s", "n_gpus": 1, "steps": 1,
        "warmup": 0, "ms_per_step": ev["model"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": "learned_plan_n50000000_d128_bf16", "held_out_cells": ev["cells"],
                   "train_records": len(train), "train_seconds_gpu_kernels": train_s},
        "fixed_rule_qps": nq / (ev["fixed"] / 1e3), "best_plan_qps": nq / (ev["best"] / 1e3),
        "latency_ms": ev,
    }
    print(json.dumps(line), flush=True)


def run_other(args):
    """--workload precision | batched: one GPU, the line carries that workload."""
    import torch

    from paper_2403_15807_gb300 import vrs
    dev = torch.device("cuda", 0)
    vrs.load()
    stream = torch.cuda.Stream(dev)
    flush = L2Flush(torch, dev)
    eng = vrs.Engine(0)
    vrs.vrs_set_option(eng.h, vrs.VRS_OPT_PROFILE, 1)
    compute = {"f32": 0, "bf16": 1, "fp8": 2}[args.compute]
    if args.workload == "precision":
        n, d, b, k = args.n or 1_000_000, args.d or 960, args.batch or 1024, args.k
        mix = gen.Mixture(d, seed=0)
        x = gen.vectors(n, mix)
        attrs = gen.attributes(n, 1, 1_000_000)
        q = gen.queries(b, mix)
        # E4M3 requests run on the bf16 copy when one is resident (its error
        # band is too wide to certify cheaply); --no-bf16-copy measures E4M3
        # storage on its own
        copies = 5 if args.no_bf16_copy else 7
        eng.load(x, attrs, dtype=vrs.VRS_F32, copies=copies)
        preds = [gen.pred_less_than(int(args.sel * 1_000_000)) if args.sel < 1 else gen.pred_all()]
        ks = np.int32([k])
        name = f"precision_n{n}_d{d}_b{b}_s{args.sel:g}_k{k}_{args.compute}"
        storage = "f32 master + e4m3 copy" if args.no_bf16_copy else "f32 master + bf16 + e4m3 copies"
    else:
        n, d, b = args.n or 10_000_000, args.d or 96, args.batch or 4096
        mix = gen.Mixture(d, seed=0)
        xb = np.empty((n, d), dtype=np.uint16)
        for off, xc in gen.vectors_chunks(n, mix):
            t = torch.from_numpy(xc).to(torch.bfloat16)
            xb[off:off + xc.shape[0]] = t.view(torch.int16).numpy().view(np.uint16)
        del t
        attrs = gen.attributes(n, 2, 1_000_000)
        q = gen.to_bf16_values(gen.queries(b, mix))
        vrs.vrs_load_vectors(eng.h, xb, dtype=vrs.VRS_BF16, copies=1 << vrs.VRS_BF16)
        for c in range(2):
            vrs.vrs_load_attribute(eng.h, c, attrs[c])
        if not args.no_grid:
            # the two predicate columns' grid, built with the table (an index)
            t0 = time.perf_counter()
            vrs.vrs_build_grid(eng.h, 0, 1)
            grid_s = time.perf_counter() - t0
        x = None
        preds, _ = gen.per_query_preds(b)
        ks = gen.per_query_k(b)
        compute = 1
        name = f"batched_n{n}_d{d}_b{b}_perquery_pred_k1-10-100_bf16"
        storage = "bf16" if args.no_grid else "bf16 + clustered copy by a 2-D grid of the two predicate columns"
    qd = torch.from_numpy(q).to(dev)
    torch.cuda.synchronize()
    clocks = Clocks(0)
    with clocks:
        times, dist_ms, launches, stages, _ = time_steps(
            torch, vrs, eng, qd, None, None, vrs.VRS_L2, args.steps, args.warmup, flush, stream,
            compute=compute, preds=preds, ks=ks)
    total_ms = sum(times)
    value = b * args.steps / (total_ms / 1e3)
    extra = {}
    # how the timed batches' queries were certified exact (first pass,
    # in-merge widening, wider tensor pass, exact GEMV)
    cert = vrs.vrs_last_cert(eng.h)
    plan = ["gemv", "compact_gemm", "mask_gemm", "cells"][vrs.vrs_last_plan(eng.h)]
    # algorithmic flops of the distance pass
    if args.workload == "precision":
        _, selected = vrs.vrs_eval_predicate(eng.h, preds[0], n)
        flops = 2.0 * b * selected * d
    else:
        sel = []
        for p in preds[:256]:
            _, c = vrs.vrs_eval_predicate(eng.h, p, n)
            sel.append(c)
        flops = 2.0 * b * float(np.mean(sel)) * d
        extra["dense_flops_per_step"] = 2.0 * b * n * d
        # the same queries, one pass per query (sample of 128)
        vrs.vrs_set_option(eng.h, vrs.VRS_OPT_BATCHED, 0)
        m = 128
        tq, _, _, _, _ = time_steps(torch, vrs, eng, qd[:m].contiguous(), None, None, vrs.VRS_L2,
                                    2, 1, flush, stream, compute=compute, preds=preds[:m],
                                    ks=ks[:m])
        extra["per_query_launch_qps"] = m * len(tq) / (sum(tq) / 1e3)
        vrs.vrs_set_option(eng.h, vrs.VRS_OPT_BATCHED, 1)
        if not args.no_grid:
            extra["grid_build_s"] = grid_s
            # the batched mask plan on the same batch (every query against
            # every row), for comparison
            vrs.vrs_set_option(eng.h, vrs.VRS_OPT_CELL_PLAN, 0)
            tm, _, _, _, _ = time_steps(torch, vrs, eng, qd, None, None, vrs.VRS_L2, 1, 1, flush,
                                        stream, compute=compute, preds=preds, ks=ks)
            extra["mask_plan_qps"] = b * len(tm) / (sum(tm) / 1e3)
            vrs.vrs_set_option(eng.h, vrs.VRS_OPT_CELL_PLAN, 1)
    ran = "bf16"
    if args.workload == "precision":
        ran = "bf16" if args.compute == "fp8" and not args.no_bf16_copy else args.compute
    if ran != args.compute:
        extra["requested_dtype"] = args.compute
    peak, src = tensor_peak({"f32": 0, "bf16": 1, "fp8": 2}[ran])
    avg = statistics.mean(dist_ms) / 1e3
    ach = flops / avg / 1e12
    line = {
        "metric": "filtered exact top-k queries/s (recall@k=1.0)",
        "value": value, "unit": "queries/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": ran,
        "data": "synthetic",
        "config": {"workload": name, "n": n, "d": d, "batch": b, "storage": storage,
                   "l2": "flushed before every step (256 MiB write, then 256 MiB read)"},
        "roofline": {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                     "frac": ach / peak, "peak_source": src, "traffic": None,
                     "kernel": ("cells_gemm_kernel" if args.workload == "batched" and not args.no_grid
                                else "umma_scan_kernel"),
                     "algorithmic_flops_per_launch": flops,
                     "avg_launch_ms": avg * 1e3},
        "stage_ms_per_step": {a: v / args.steps for a, v in stages.items()},
        "gpu_launches": int(launches),
        "certificate": cert,
        "plan": plan,
    }
    line.update(extra)
    cs = clocks.summary()
    if cs:
        line["clocks"] = cs
    print(json.dumps(line), flush=True)
    eng.close()


def run_next(args):
    """Range search, vector join and disjunctions on the 1M x 128 fp32 table
    (10 % of its rows selected), one GPU, L2 flushed before every call.
    range: 16 queries, the bound near each query's 100th neighbour; join: a
    100k-row query relation with 10 % of its rows selected, top-10 each
    (--compute f32 or bf16); dnf: 16 queries under a 4-value IN-list."""
    import torch

    from paper_2403_15807_gb300 import vrs
    dev = torch.device("cuda", 0)
    vrs.load()
    flush = L2Flush(torch, dev)
    n, d, b, k = args.n or 1_000_000, args.d or 128, args.batch or 16, args.k
    mix = gen.Mixture(d, seed=0)
    x = gen.vectors(n, mix)
    attrs = gen.attributes(n, 1, 1000)
    eng = vrs.Engine(0)
    eng.load(x, attrs, dtype=vrs.VRS_F32, copies=3)
    del x
    pred = gen.pred_less_than(100)
    stream = torch.cuda.Stream(dev)
    times, extra = [], {}
    if args.workload == "range":
        qd = torch.from_numpy(gen.queries(b, mix)).to(dev)
        _, dist = eng.query(qd, [pred], np.int32([100]))
        eps = float(dist[:, 99].median())
        for i in range(args.warmup + args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            offs, _, _ = eng.range_query(qd, pred, eps)
            torch.cuda.synchronize()
            if i >= args.warmup:
                times.append(time.perf_counter() - t0)
        units, name = b, f"range_n{n}_d{d}_b{b}_s0.1_eps100th_l2"
        extra["results_per_query"] = float(offs[-1]) / b
        compute = "f32"
    elif args.workload == "join":
        m = 100_000
        qrel = torch.from_numpy(gen.queries(m, mix)).to(dev)
        qattrs = torch.from_numpy(gen.attributes(m, 1, 1000, seed=1)).to(dev)
        cd = vrs.VRS_F32 if args.compute == "f32" else vrs.VRS_BF16
        for i in range(args.warmup + args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            qids, _, _ = eng.join_topk(qrel, qattrs, gen.Pred([0], [0], [100]), pred, k,
                                       compute=cd)
            torch.cuda.synchronize()
            if i >= args.warmup:
                times.append(time.perf_counter() - t0)
        units, name = int(qids.size), f"join_q{m}_s0.1_n{n}_d{d}_s0.1_k{k}_{args.compute}"
        compute = args.compute if args.compute != "fp8" else "bf16"
    else:
        qd = torch.from_numpy(gen.queries(b, mix)).to(dev)
        conjs = vrs.in_list(0, [3, 30, 300, 600])
        for i in range(args.warmup + args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                e0.record(stream)
                vrs.vrs_query_dnf(eng.h, qd, conjs, k, stream=stream)
                e1.record(stream)
            stream.synchronize()
            if i >= args.warmup:
                times.append(e0.elapsed_time(e1) / 1e3)
        units, name = b, f"dnf_inlist4_n{n}_d{d}_b{b}_k{k}_l2"
        compute = "f32"
    total = sum(times)
    line = {
        "metric": "filtered exact queries/s" if args.workload != "join"
                  else "filtered exact top-k query rows/s",
        "value": units * len(times) / total, "unit": "queries/s" if args.workload != "join"
        else "query rows/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total / len(times) * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": compute, "data": "synthetic",
        "config": {"workload": name, "n": n, "d": d,
                   "l2": "flushed before every call (256 MiB write, then 256 MiB read)"},
    }
    line.update(extra)
    print(json.dumps(line), flush=True)
    eng.close()


def max_over_ranks(dist, value: float, device) -> float:
    """The largest of every rank's `value` (the slowest rank's time decides
    the whole-job throughput); `value` itself on one rank."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, units_per_rank_step: int, steps: int, max_ms: float) -> float:
    """Whole-job units/s: every rank processes its own batch each step
    (weak scaling), all ranks finish within the slowest rank's time."""
    return world * units_per_rank_step * steps / (max_ms / 1e3)


def run_vrs(args):
    import torch

    from paper_2403_15807_gb300 import vrs

    ws, rank, local = dist_env()
    dist = None
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    vrs.load()

    wl = workload(args)
    x, attrs, q = load_inputs(wl, rank)
    metric = vrs.VRS_L2 if wl.metric == "l2" else vrs.VRS_IP
    eng = vrs.Engine(local)
    vrs.vrs_set_option(eng.h, vrs.VRS_OPT_PAIR_COPY, 0 if args.no_pair_copy else 1)
    eng.load(x, attrs)
    vrs.vrs_set_option(eng.h, vrs.VRS_OPT_PROFILE, 1)
    dist_kernel = "umma_rows_kernel" if args.no_pair_copy else DIST_KERNEL
    pred = wl.pred()
    _, selected = vrs.vrs_eval_predicate(eng.h, pred, wl.n)
    stream = torch.cuda.Stream(dev)
    flush = L2Flush(torch, dev)
    qd = torch.from_numpy(q).to(dev)

    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    wall0 = time.perf_counter()
    with clocks:
        times, dist_ms, launches, stages, _ = time_steps(
            torch, vrs, eng, qd, pred, wl.k, metric, args.steps, args.warmup, flush, stream)
    wall = time.perf_counter() - wall0
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    total_ms = max_over_ranks(dist, sum(times), dev)
    value = job_throughput(ws, wl.batch, args.steps, total_ms)

    # e2e through the C ABI with pinned host buffers: the vrs_query entry
    # point itself (arguments marshalled once; the upload of the queries, the
    # search and the download of the results inside the timed call)
    import ctypes
    qh = torch.from_numpy(q).pin_memory()
    oid_h = torch.empty((wl.batch, wl.k), dtype=torch.int64).pin_memory()
    od_h = torch.empty((wl.batch, wl.k), dtype=torch.float32).pin_memory()
    kk = np.int32([wl.k])
    parr, _keep = vrs.make_preds([pred])
    lib = vrs.load()
    c_args = (eng.h, ctypes.c_void_p(qh.data_ptr()), wl.batch, wl.d, parr, 1,
              kk.ctypes.data_as(ctypes.c_void_p), 1, wl.k, metric, 0,
              ctypes.c_void_p(oid_h.data_ptr()), ctypes.c_void_p(od_h.data_ptr()), 0, None)
    e2e_t = []
    vrs.vrs_set_option(eng.h, vrs.VRS_OPT_PROFILE, 0)   # no stage events in this loop
    for i in range(args.warmup + args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = lib.vrs_query(*c_args)
        if i >= args.warmup:
            e2e_t.append(time.perf_counter() - t0)
        if st != vrs.VRS_OK:
            raise vrs.VrsError(st, vrs.vrs_last_error())
    e2e_total = max_over_ranks(dist, sum(e2e_t), dev)
    e2e = {"value": job_throughput(ws, wl.batch, args.steps, e2e_total * 1e3), "unit": "queries/s",
           "h2d_bytes_per_step": int(wl.batch * wl.d * 4),
           "d2h_bytes_per_step": int(wl.batch * wl.k * (8 + 4))}

    peak, peak_src = measured_peak()

    def alg_bytes(selected, batch):
        # algorithmic bytes of one distance launch: the selected rows, their
        # norms and ids, and the query batch
        return selected * (wl.d * 4 + 4 + 4) + batch * wl.d * 4

    # the metric's selectivity axis at the headline batch: q/s and the
    # distance kernel's fraction of the HBM roofline per cell
    sel_sweep = None
    if not args.no_sel_sweep:
        sel_sweep = {}
        for sv in SEL_AXIS:
            pr = gen.sweep_cell(wl.batch, sv, wl.k, wl.metric, n=wl.n, d=wl.d).pred()
            _, nsel = vrs.vrs_eval_predicate(eng.h, pr, wl.n)
            tt, dm, _, st, _ = time_steps(torch, vrs, eng, qd, pr, wl.k, metric,
                                          max(5, args.steps // 2), 3, flush, stream)
            avg = statistics.mean(dm) / 1e3
            ach = alg_bytes(nsel, wl.batch) / avg / 1e9
            sel_sweep[f"s{sv:g}"] = {
                "selected_rows": int(nsel), "qps": wl.batch * len(tt) / (sum(tt) / 1e3),
                "ms_per_step": sum(tt) / len(tt),
                "distance_ms": avg * 1e3, "achieved_gbs": ach, "frac": ach / peak,
                "stage_ms": {a: round(v / len(tt), 4) for a, v in st.items()}}

    # the other axes of the scan sweep at s = 10 %: batch 1 / 256 / 1024, k = 100,
    # and inner product on unit-normalised rows (a table of its own)
    axes = None
    if not args.no_sel_sweep and rank == 0:
        axes = {}
        pr10 = gen.sweep_cell(wl.batch, 0.1, wl.k, wl.metric, n=wl.n, d=wl.d).pred()

        def cell(e, qq, kk, m):
            tt, _, _, _, _ = time_steps(torch, vrs, e, qq, pr10, kk, m, 5, 3, flush, stream)
            return {"qps": qq.shape[0] * len(tt) / (sum(tt) / 1e3), "ms_per_step": sum(tt) / len(tt)}

        for bb in (1, 256, 1024):
            qb = torch.from_numpy(gen.queries(bb, wl.mixture(), unit=wl.unit)).to(dev)
            axes[f"b{bb}_s0.1_k{wl.k}_{wl.metric}"] = cell(eng, qb, wl.k, metric)
        axes[f"b{wl.batch}_s0.1_k100_{wl.metric}"] = cell(eng, qd, 100, metric)
        if wl.metric == "l2":
            xu = gen.vectors(wl.n, wl.mixture(), unit=True)
            qu = torch.from_numpy(gen.queries(wl.batch, wl.mixture(), unit=True)).to(dev)
            with vrs.Engine(local) as eu:
                vrs.vrs_set_option(eu.h, vrs.VRS_OPT_PAIR_COPY, 0 if args.no_pair_copy else 1)
                eu.load(xu, attrs)
                axes[f"b{wl.batch}_s0.1_k{wl.k}_ip_unit"] = cell(eu, qu, wl.k, vrs.VRS_IP)
            del xu

    sweep = None
    if args.sweep:
        sweep = {}
        for b in (1, 16, 256, 1024):
            qb = torch.from_numpy(gen.queries(b, wl.mixture(), unit=wl.unit)).to(dev)
            for s in (0.001, 0.01, 0.1, 0.5, 1.0):
                pr = gen.sweep_cell(b, s, wl.k, wl.metric, n=wl.n, d=wl.d).pred()
                tt, _, _, st, _ = time_steps(torch, vrs, eng, qb, pr, wl.k, metric, 3, 2, flush,
                                             stream)
                sweep[f"b{b}_s{s:g}"] = {"qps": b * len(tt) / (sum(tt) / 1e3),
                                         "stage_ms": {a: round(v / len(tt), 4) for a, v in st.items()}}

    if rank == 0:
        alg = alg_bytes(selected, wl.batch)
        avg_dist_s = statistics.mean(dist_ms) / 1e3
        achieved = alg / avg_dist_s / 1e9
        cell = wl.name
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "peak_source": peak_src,
                    "traffic": recorded_traffic(dist_kernel, cell),
                    "kernel": dist_kernel,
                    "algorithmic_bytes_per_launch": int(alg),
                    "avg_launch_ms": avg_dist_s * 1e3}
        line = {
            "metric": "filtered exact top-k queries/s (recall@k=1.0)",
            "value": value, "unit": "queries/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": dict(config_of(wl, args), parallelism=f"independent query batches x{ws}",
                           selected_rows=int(selected)),
            "e2e": e2e,
            "roofline": roofline,
            "stage_ms_per_step": {a: v / args.steps for a, v in stages.items()},
            "gpu_launches": int(launches),
            "wall_s_timed_region": wall,
        }
        cs = clocks.summary()
        if cs:
            line["clocks"] = cs
        if sel_sweep:
            line["sweep"] = {"axis": "selectivity", "batch": wl.batch, "cells": sel_sweep,
                             "roofline_peak_gbs": peak, "peak_source": peak_src}
        if axes:
            line["axes"] = {"selectivity": 0.1, "note": "batch, k and metric axes of the scan sweep",
                            "cells": axes}
        if sweep:
            line["sweep_qps"] = sweep
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(wl, x, attrs, q, args.cpu_seconds)
        print(json.dumps(line), flush=True)
    eng.close()
    if dist:
        dist.destroy_process_group()


def run_sharded(args):
    """Row-sharded search: rank r holds rows [r n / W, (r + 1) n / W) of the
    table, every rank answers the same query batch, the ranks all-gather
    their [batch x k] lists (NCCL) and each merges them on its GPU.  The
    whole job processes one batch per step (strong scaling); value = batch
    x steps / the slowest rank's time."""
    import torch

    from paper_2403_15807_gb300 import shards, vrs

    ws, rank, local = dist_env()
    dist = None
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    vrs.load()
    wl = workload(args)
    x, attrs, q = load_inputs(wl, 0)
    lo, hi = shards.shard_rows(wl.n, ws, rank)
    metric = vrs.VRS_L2 if wl.metric == "l2" else vrs.VRS_IP
    eng = vrs.Engine(local)
    vrs.vrs_set_option(eng.h, vrs.VRS_OPT_PAIR_COPY, 1)
    eng.load(np.ascontiguousarray(x[lo:hi]), np.ascontiguousarray(attrs[:, lo:hi]))
    offsets = shards.row_offsets(wl.n, ws)
    pred = wl.pred()
    _, local_sel = vrs.vrs_eval_predicate(eng.h, pred, hi - lo)
    selected = shards.global_count(dist, local_sel, dev) if dist else local_sel
    flush = L2Flush(torch, dev)
    qd = torch.from_numpy(q).to(dev)
    kk = np.int32([wl.k])
    stream = torch.cuda.current_stream(dev)

    def step():
        ids, dd = vrs.vrs_query(eng.h, qd, [pred], kk, k_max=wl.k, metric=metric, stream=stream)
        if dist:
            ia, da = shards.gather_topk(dist, ids, dd)
            ids, dd = shards.merge(vrs, ia, da, offsets, metric, stream=stream)
        return ids, dd

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    with clocks:
        for i in range(args.warmup + args.steps):
            flush.zero_()
            j = i - args.warmup
            if j >= 0:
                ev[j][0].record(stream)
            out = step()
            if j >= 0:
                ev[j][1].record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    total_ms = max_over_ranks(dist, sum(a.elapsed_time(b) for a, b in ev), dev)
    if rank == 0:
        line = {
            "metric": "filtered exact top-k queries/s (recall@k=1.0)",
            "value": wl.batch * args.steps / (total_ms / 1e3), "unit": "queries/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(config_of(wl, args), parallelism=f"row shards x{ws}",
                           selected_rows=int(selected)),
            # per step: the query's three kernels (filter, distance, merge) and
            # the shard merge when there is more than one shard
            "gpu_launches": args.steps * (3 + (1 if dist else 0)),
        }
        cs = clocks.summary()
        if cs:
            line["clocks"] = cs
        print(json.dumps(line), flush=True)
    eng.close()
    if dist:
        dist.destroy_process_group()


def run_peaks(args):
    """Dense matrix-multiply peaks of this GPU through cuBLAS (PyTorch), for
    the roofline denominators the driver does not measure: FP32 without
    TF32 (the FFMA pipe), TF32, BF16 and FP8 E4M3 (per-tensor scales).
    8192^3 products, CUDA events over 20 repetitions after 5 warm-ups."""
    import torch
    dev = torch.device("cuda", 0)
    n = 8192
    out = {}

    def timed(fn, flops):
        for _ in range(5):
            fn()
        st, en = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        st.record()
        for _ in range(20):
            fn()
        en.record()
        torch.cuda.synchronize()
        return flops * 20 / (st.elapsed_time(en) / 1e3) / 1e12

    flops = 2.0 * n ** 3
    a32 = torch.randn(n, n, device=dev)
    b32 = torch.randn(n, n, device=dev)
    torch.backends.cuda.matmul.allow_tf32 = False
    out["fp32_ffma_tflops"] = timed(lambda: a32 @ b32, flops)
    torch.backends.cuda.matmul.allow_tf32 = True
    out["tf32_tflops"] = timed(lambda: a32 @ b32, flops)
    torch.backends.cuda.matmul.allow_tf32 = False
    a16, b16 = a32.to(torch.bfloat16), b32.to(torch.bfloat16)
    out["bf16_tflops"] = timed(lambda: a16 @ b16, flops)
    try:
        a8 = a32.to(torch.float8_e4m3fn)
        b8 = b32.to(torch.float8_e4m3fn).t()
        one = torch.ones((), device=dev)
        out["fp8_e4m3_tflops"] = timed(
            lambda: torch._scaled_mm(a8, b8, scale_a=one, scale_b=one, out_dtype=torch.bfloat16),
            flops)
    except Exception as exc:   # not every PyTorch build exposes it
        out["fp8_e4m3_tflops"] = None
        out["fp8_error"] = str(exc)[:120]
    clocks = Clocks(0)
    with clocks:
        timed(lambda: a16 @ b16, flops)
    del a32, b32, a16, b16
    line = {"metric": "dense matmul peak (cuBLAS)", "unit": "TFLOP/s", "n": n,
            "results": out, "clocks": clocks.summary(), "gather": gather_ceiling(torch, dev)}
    print(json.dumps(line), flush=True)


def gather_ceiling(torch, dev):
    """The distance pass's memory access alone: every listed row of a 1M x 128
    float32 table (512-byte rows) read once in full by the library's
    measurement kernel (vrs_probe_gather), for the ids of 10 % of the rows in
    ascending order and for every row; CUDA events, L2 flushed before each of
    25 repetitions, median of the last 20.  An empty launch gives the fixed
    cost that any event-timed launch carries."""
    from paper_2403_15807_gb300 import vrs
    vrs.load()
    flush = L2Flush(torch, dev)
    n, d = 1_000_000, 128
    gen_ = torch.Generator(device="cpu").manual_seed(0)
    X = torch.rand(n, d, generator=gen_).to(dev)
    hbm, _ = measured_peak()
    res = {}
    for name, m in (("empty", 0), ("s0.1", n // 10), ("s1", n)):
        if m == n:
            ids = torch.arange(n, dtype=torch.int32, device=dev)
        else:
            ids = torch.randperm(n, generator=gen_)[:m].sort().values.to(torch.int32).to(dev)
        acc = torch.zeros(1, dtype=torch.float32, device=dev)
        ts = []
        for _ in range(25):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            vrs.vrs_probe_gather(X, ids, acc)
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        ms = statistics.median(ts[5:])
        cell = {"rows": m, "bytes": m * d * 4, "ms": ms}
        if m:
            gbs = m * d * 4 / (ms / 1e3) / 1e9
            ref = float(X[ids.long()].double().sum()) * 25
            cell.update({"gbs": gbs, "frac_of_measured_hbm": gbs / hbm,
                         "sum_rel_err": abs(float(acc) - ref) / ref})
        res[name] = cell
    return res


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "learned":
        run_learned(args)
    elif args.workload == "peaks":
        run_peaks(args)
    elif args.workload in ("range", "join", "dnf"):
        run_next(args)
    elif args.workload != "sweep":
        run_other(args)
    elif args.shard == "rows":
        run_sharded(args)
    else:
        run_vrs(args)


if __name__ == "__main__":
    main()
