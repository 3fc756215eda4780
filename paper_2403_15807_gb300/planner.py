"""Learned access-path selection for the scan (the optimizer the paper's
Sec. 5.2 / 5.3 takeaways ask for: the choice depends on selectivity,
dimensionality and batch size).

The model is the library's 6 -> 64 -> 64 -> 3 network (include/vrs.h,
vrs_mlp_*): from (ln N, ln d, ln batch, ln selectivity, ln k, bytes per
element) it predicts the standardised ln(latency) of the three scan plans
GEMV, COMPACT_GEMM and MASK_GEMM.  Everything here is orchestration: the
timings come from the engine itself (each plan forced in turn, CUDA events on
the query stream), and training and inference run in the library's kernels.

    records = timing_grid(...)            # measure plans on a grid
    model = fit(records)                  # GPU training (vrs_mlp_train)
    write_planner(path, model)            # file for vrs_planner_load
"""
from __future__ import annotations

import dataclasses
import json
import math
import struct
from typing import Dict, List, Optional, Sequence

import numpy as np

from . import vrs

PLANS = ("gemv", "compact_gemm", "mask_gemm")
PLAN_IDS = (vrs.VRS_PLAN_GEMV, vrs.VRS_PLAN_COMPACT_GEMM, vrs.VRS_PLAN_MASK_GEMM)
BPE = {"f32": 4.0, "bf16": 2.0, "fp8": 1.0}
DTYPE_ID = {"f32": vrs.VRS_F32, "bf16": vrs.VRS_BF16, "fp8": vrs.VRS_FP8E4M3}
# plans each compute dtype supports (GEMV reads float32 or bf16 rows; the
# tensor plans read bf16 or E4M3 operands)
AVAILABLE = {"f32": (True, False, False), "bf16": (True, True, True), "fp8": (False, True, True)}


def features(n, d, b, s, k, dtype) -> List[float]:
    return [math.log(n), math.log(d), math.log(b), math.log(max(s, 1e-6)), math.log(max(k, 1)),
            BPE[dtype]]


@dataclasses.dataclass
class Model:
    params: np.ndarray          # float32 [4803]
    fmean: np.ndarray           # [6]
    fstd: np.ndarray            # [6]
    omean: float
    ostd: float

    def predict(self, feats: np.ndarray, bf16: bool = True) -> np.ndarray:
        """Predicted ln(ms) [m x 3] with the library's inference kernel."""
        x = (np.asarray(feats, np.float32) - self.fmean) / self.fstd
        y = vrs.vrs_mlp_forward(self.params, x, bf16=bf16)
        return y * self.ostd + self.omean

    def choose(self, feats: np.ndarray, dtypes: Sequence[str]) -> np.ndarray:
        y = self.predict(feats)
        out = np.empty(len(dtypes), np.int64)
        for i, dt in enumerate(dtypes):
            yy = np.where(np.asarray(AVAILABLE[dt]), y[i], np.inf)
            out[i] = int(np.argmin(yy))
        return out


def _fnv1a(data: bytes) -> int:
    h = 1469598103934665603
    for c in data:
        h ^= c
        h = (h * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def write_planner(path: str, m: Model) -> None:
    """The file format vrs_planner_load reads (see include/vrs.h)."""
    body = b"VRSPLAN1" + struct.pack("<II", 1, m.params.size)
    body += np.asarray(m.fmean, "<f4").tobytes() + np.asarray(m.fstd, "<f4").tobytes()
    body += struct.pack("<ff", float(m.omean), float(m.ostd))
    body += np.asarray(m.params, "<f4").tobytes()
    with open(path, "wb") as f:
        f.write(body + struct.pack("<Q", _fnv1a(body)))


def read_planner(path: str) -> Model:
    """Parse a planner file (checksum verified)."""
    blob = open(path, "rb").read()
    body, ck = blob[:-8], struct.unpack("<Q", blob[-8:])[0]
    if body[:8] != b"VRSPLAN1" or _fnv1a(body) != ck:
        raise ValueError(f"{path}: not a valid planner file")
    ver, n = struct.unpack("<II", body[8:16])
    f = np.frombuffer(body[16:16 + 56], "<f4")
    params = np.frombuffer(body[72:72 + 4 * n], "<f4").astype(np.float32)
    return Model(params, f[:6].copy(), f[6:12].copy(), float(f[12]), float(f[13]))


def fixed_rule(dtype: str, s: float) -> int:
    """The engine's rule without a model: FP32 -> GEMV; reduced precision ->
    COMPACT_GEMM below 30 % selectivity (20 % for FP8), MASK_GEMM above."""
    if dtype == "f32":
        return 0
    return 2 if s >= (0.2 if dtype == "fp8" else 0.3) else 1


# ---------------------------------------------------------------- data

def to_arrays(records: List[dict]):
    """Features [m x 6], targets ln(ms) [m x 3] and mask [m x 3]."""
    X = np.array([features(r["n"], r["d"], r["b"], r["s"], r["k"], r["dtype"]) for r in records],
                 np.float32)
    T = np.zeros((len(records), 3), np.float32)
    M = np.zeros((len(records), 3), np.float32)
    for i, r in enumerate(records):
        for p, name in enumerate(PLANS):
            ms = r["ms"].get(name)
            if ms is not None and math.isfinite(ms) and ms > 0:
                T[i, p] = math.log(ms)
                M[i, p] = 1.0
    return X, T, M


def fit(records: List[dict], steps: int = 3000, lr: float = 3e-3, seed: int = 0) -> Model:
    """Train the network on measured timings with the library's kernels."""
    X, T, M = to_arrays(records)
    fmean, fstd = X.mean(0), X.std(0)
    fstd[fstd == 0] = 1.0
    tv = T[M > 0]
    omean, ostd = float(tv.mean()), float(tv.std() or 1.0)
    Xs = (X - fmean) / fstd
    Ts = np.where(M > 0, (T - omean) / ostd, 0.0).astype(np.float32)
    rng = np.random.default_rng(seed)
    n = vrs.vrs_mlp_nparams()
    p = np.zeros(n, np.float32)
    # He-style initialisation per layer
    sizes = [(64, 6), (64,), (64, 64), (64,), (3, 64), (3,)]
    off = 0
    for sh in sizes:
        cnt = int(np.prod(sh))
        if len(sh) == 2:
            p[off:off + cnt] = rng.standard_normal(cnt) * math.sqrt(2.0 / sh[1])
        off += cnt
    params, loss = vrs.vrs_mlp_train(p, Xs, Ts, M, steps, lr)
    return Model(params, fmean.astype(np.float32), fstd.astype(np.float32), omean, ostd)


# ---------------------------------------------------------------- timing grid

def time_plan(eng, q, pred, k, plan, dtype, reps: int = 2) -> float:
    """Median device time (ms) of the whole query with `plan` forced."""
    import torch
    vrs.vrs_set_plan(eng.h, plan)
    kk = np.int32([k])
    out = []
    for i in range(reps + 1):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        vrs.vrs_query(eng.h, q, [pred], kk, compute=DTYPE_ID[dtype])
        ev1.record()
        torch.cuda.synchronize()
        if i:
            out.append(ev0.elapsed_time(ev1))
    vrs.vrs_set_plan(eng.h, vrs.VRS_PLAN_AUTO)
    return float(np.median(out))


def work_estimate(n, d, b, s, plan, dtype) -> float:
    """Rough flop count of a cell, used only to skip cells that would take
    seconds (those plans are recorded as not measured)."""
    rows = n if plan == 2 else n * s
    return 2.0 * b * rows * d


def timing_grid(eng, n: int, d: int, mix, batches=(1, 16, 256, 4096),
                sels=(1e-4, 1e-2, 0.1, 0.5, 1.0), ks=(10, 100), dtypes=("bf16", "fp8", "f32"),
                attr_range: int = 1_000_000, budget_flops: float = 4e12,
                gemv_budget_flops: float = 2e11, log=None) -> List[dict]:
    """Measure every available plan on every cell of the grid (the engine
    must hold the table with float32, bf16 and E4M3 copies and an attribute
    column 0 uniform on [0, attr_range))."""
    import torch

    import gen
    recs = []
    for b in batches:
        q = torch.from_numpy(gen.queries(b, mix)).cuda()
        for s in sels:
            pred = gen.pred_less_than(int(round(s * attr_range))) if s < 1 else gen.pred_all()
            for k in ks:
                for dt in dtypes:
                    r = {"n": n, "d": d, "b": b, "s": s, "k": k, "dtype": dt, "ms": {}}
                    for p, name in enumerate(PLANS):
                        if not AVAILABLE[dt][p]:
                            continue
                        w = work_estimate(n, d, b, s, p, dt)
                        lim = gemv_budget_flops if p == 0 else budget_flops
                        if w > lim:
                            r["ms"][name] = None
                            continue
                        try:
                            r["ms"][name] = time_plan(eng, q, pred, k, PLAN_IDS[p], dt)
                        except vrs.VrsError:
                            r["ms"][name] = None
                    recs.append(r)
                    if log:
                        log(json.dumps(r))
    return recs


def evaluate(model: Optional[Model], records: List[dict]) -> Dict[str, float]:
    """Total latency of the plans chosen by the model, by the fixed rule and
    by an oracle that knows every measured latency (cells where every plan the
    model could choose was measured)."""
    X, T, M = to_arrays(records)
    dts = [r["dtype"] for r in records]
    lat = np.where(M > 0, np.exp(T), np.inf)
    choose = model.choose(X, dts) if model is not None else None
    tot = {"model": 0.0, "fixed": 0.0, "best": 0.0, "cells": 0}
    for i, r in enumerate(records):
        avail = np.array(AVAILABLE[r["dtype"]]) & (M[i] > 0)
        if avail.sum() < 1 or not np.all(M[i][np.array(AVAILABLE[r["dtype"]])] > 0):
            continue
        f = fixed_rule(r["dtype"], r["s"])
        tot["fixed"] += lat[i, f]
        tot["best"] += lat[i][avail].min()
        if choose is not None:
            tot["model"] += lat[i, choose[i]]
        tot["cells"] += 1
    return {k: (int(v) if k == "cells" else float(v)) for k, v in tot.items()}


def split_50m(grid: List[dict], table: List[dict], held_batches=(4, 64, 1024)):
    """Evaluation protocol at N = 5e7, d = 128 (bf16 rows): train on the
    timing grid plus the 5e7-row cells at the grid's batch sizes; test on the
    5e7-row cells at the batch sizes the training never saw."""
    train = list(grid) + [r for r in table if r["b"] not in held_batches]
    test = [r for r in table if r["b"] in held_batches]
    return train, test


# ---------------------------------------------------------------- command line

GRID_TABLES = ((100_000, 64), (100_000, 384), (1_000_000, 128), (1_000_000, 384),
               (1_000_000, 960), (10_000_000, 64), (10_000_000, 128))


def _grid_main(out: str, tables=GRID_TABLES) -> None:
    """Timing grid over several tables (float32 master + bf16 + E4M3)."""
    import gen
    recs = []
    for n, d in tables:
        mix = gen.Mixture(d, seed=0)
        x = gen.vectors(n, mix)
        attrs = gen.attributes(n, 1, 1_000_000)
        with vrs.Engine(0) as e:
            e.load(x, attrs, dtype=vrs.VRS_F32, copies=7)
            del x
            recs += timing_grid(e, n, d, mix, log=print)
        with open(out, "w") as f:
            json.dump({"device": "GB300", "records": recs}, f)


def _eval_main(out: str, n: int = 50_000_000, d: int = 128) -> None:
    """Evaluation table: bf16-stored rows, every plan measured per cell."""
    import torch

    import gen
    mix = gen.Mixture(d, seed=0)
    xb = np.empty((n, d), np.uint16)
    for off, xc in gen.vectors_chunks(n, mix):
        xb[off:off + xc.shape[0]] = torch.from_numpy(xc).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    attrs = gen.attributes(n, 1, 1_000_000)
    with vrs.Engine(0) as e:
        vrs.vrs_load_vectors(e.h, xb, dtype=vrs.VRS_BF16, copies=1 << vrs.VRS_BF16)
        del xb
        vrs.vrs_load_attribute(e.h, 0, attrs[0])
        recs = timing_grid(e, n, d, mix, batches=(1, 4, 16, 64, 256, 1024, 4096),
                           sels=(1e-4, 1e-3, 1e-2, 0.1, 0.5, 1.0), ks=(10, 100),
                           dtypes=("bf16",), budget_flops=6e13, gemv_budget_flops=4e12,
                           log=print)
    with open(out, "w") as f:
        json.dump({"device": "GB300", "records": recs}, f)


def _train_main(data: str, out: str, steps: int) -> None:
    with open(data) as f:
        recs = json.load(f)["records"]
    m = fit(recs, steps=steps)
    write_planner(out, m)
    print(json.dumps(evaluate(m, recs)))


if __name__ == "__main__":
    import argparse
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    ap = argparse.ArgumentParser(description="timing grid / training of the plan model")
    ap.add_argument("cmd", choices=["grid", "eval", "train", "score"])
    ap.add_argument("--model")
    ap.add_argument("--out", required=True)
    ap.add_argument("--data")
    ap.add_argument("--steps", type=int, default=3000)
    a = ap.parse_args()
    vrs.load()
    if a.cmd == "grid":
        _grid_main(a.out)
    elif a.cmd == "eval":
        _eval_main(a.out)
    elif a.cmd == "train":
        _train_main(a.data, a.out, a.steps)
    else:
        # total latency of model / fixed-rule / best plans on a timing table
        with open(a.data) as f:
            recs = json.load(f)["records"]
        res = evaluate(read_planner(a.model), recs)
        with open(a.out, "w") as f:
            json.dump(res, f)
        print(json.dumps(res))
