#!/usr/bin/env python
"""Benchmark of the DDF hot path on one GB300 (or N independent replicas).

One step = the whole path over the workload "lap7_128+elast3x3_64" (a 3-D
7-point Laplacian on a 128^3 grid and a 3x3-block elasticity matrix on a 27-point
stencil over 64^3 nodes): for each matrix A and its lower triangle L,
    ddf_inspect(A, SpMV) -> ddf_spmv -> ddf_inspect(L, SpTRSV) -> ddf_sptrsv
with CSR inputs and vectors already resident in HBM.  ``value`` is the
executors' algorithmic bytes (plan statistics) moved per second of the whole
step, inspection included.  Extra keys report each phase on its own.

``--impl reference`` times the CPU oracle (plain sequential C, FP64) on the
host cores over the same workload and prints the same line with
``"impl": "reference"``.
"""
from __future__ import annotations

import argparse
import json
import threading
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "SpMV & SpTRSV GB/s as % of HBM roofline; mixed-precision vs FP64 speedup"
WORKLOAD = ("lap7_128", "elast3x3_64")
L2_FLUSH_BYTES = 256 << 20
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=float, default=1.0, help="grid scale (1.0 = the full workload)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-critical-path", action="store_true", help="skip the chain solve that measures t_hop")
    ap.add_argument("--streams", type=int, default=4, choices=[1, 2, 4],
                    help="1: everything on one stream; 2: one stream and host thread per matrix; "
                         "4 (default): one per chain, inspect(A)+spmv and inspect(L)+sptrsv of each matrix")
    ap.add_argument("--serial", action="store_true", help="same as --streams 1")
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--coarsen", type=int, default=None,
                    help="SpTRSV rows per block (coarsen_rows; 0 = plain level sets; default: library default)")
    a = ap.parse_args()
    if a.serial:
        a.streams = 1
    return a


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def build_inputs(scale):
    mats = []
    for name in WORKLOAD:
        a, lo, x, b = synth.workload(name, scale)
        mats.append((name, a, lo, x, b))
    return mats


def csr_bytes(m):
    return 4 * (m.n_rows + 1) + 12 * m.nnz


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
class L2Flush:
    """Between timed iterations: write a buffer larger than L2, then read
    another one, so that the written lines are written back to DRAM here and
    not during the timed work that follows (which then starts on a cold L2
    holding clean lines only)."""

    def __init__(self, torch, dev):
        self.w = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
        self.r = torch.ones(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)

    def __call__(self):
        self.w.zero_()
        self.r.sum()


def aggregate(ms, exec_b, world, dev):
    """Whole-job figures over `world` replicas: the step time is the maximum
    over ranks, the value the bytes of all ranks over that time (GB/s)."""
    if world > 1:
        import torch
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    return ms, exec_b * world / (ms * 1e-3) / 1e9


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_2111_12243_gb300 as ddf
    from paper_2111_12243_gb300 import build as ddf_build

    ddf_build.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()
    mats = build_inputs(args.scale)

    def to_dev(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    D = []
    for name, a, lo, x, b in mats:
        D.append({
            "name": name, "a": a, "lo": lo,
            "A": (to_dev(a.rowptr), to_dev(a.colidx), to_dev(a.values)),
            "L": (to_dev(lo.rowptr), to_dev(lo.colidx), to_dev(lo.values)),
            "x": to_dev(x), "b": to_dev(b),
            "y": torch.empty(a.n_rows, dtype=torch.float64, device=dev),
            "xs": torch.empty(lo.n_rows, dtype=torch.float64, device=dev),
        })
    flush = L2Flush(torch, dev)
    phases = ("inspect_spmv", "spmv", "inspect_sptrsv", "sptrsv")

    opts_L = ddf.ddf_opts_default(coarsen_rows=args.coarsen) if args.coarsen is not None else None

    def chain_a(d, s, e, rec, out, i):
        """inspect(A) and spmv of one matrix on stream s (events e[0..2])."""
        torch.cuda.set_device(dev)
        e[0].record(s)
        pA = ddf.ddf_inspect(*d["A"], d["a"].n_cols, ddf.DDF_SPMV, None, s)
        e[1].record(s)
        ddf.ddf_spmv(pA, d["x"], d["y"], stream=s)
        e[2].record(s)
        if rec:
            out[i][0] = ddf.ddf_plan_stats(pA)
        pA.destroy()

    def chain_l(d, s, e, rec, out, i):
        """inspect(L) and sptrsv of one matrix on stream s (events e[3..5])."""
        torch.cuda.set_device(dev)
        e[3].record(s)
        pL = ddf.ddf_inspect(*d["L"], d["lo"].n_cols, ddf.DDF_SPTRSV, opts_L, s)
        e[4].record(s)
        ddf.ddf_sptrsv(pL, d["b"], d["xs"], stream=s)
        e[5].record(s)
        if rec:
            out[i][1] = ddf.ddf_plan_stats(pL)
        pL.destroy()

    def one(d, s, e, rec, out, i):
        chain_a(d, s, e, rec, out, i)
        chain_l(d, s, e, rec, out, i)

    # Larger matrices have the longer pipelines: their streams get the higher
    # priority, the others fill the SMs they leave idle.
    order = sorted(range(len(D)), key=lambda i: -(D[i]["a"].nnz + D[i]["lo"].nnz))
    lo_p, hi_p = torch.cuda.Stream.priority_range() if hasattr(torch.cuda.Stream, "priority_range") else (0, -1)
    prio = {i: (hi_p if k == 0 else lo_p) for k, i in enumerate(order)}
    side = [torch.cuda.Stream(device=dev, priority=prio[i]) for i in range(len(D))]
    side_l = [torch.cuda.Stream(device=dev, priority=prio[i]) for i in range(len(D))]

    def step(record):
        """One step; returns per-matrix phase events, plan stats and the step's
        start / end events on the main stream.  --streams 1: matrices and their
        two chains one after another on the main stream; 2: one stream and host
        thread per matrix; 4: one per chain (inspect(A) + spmv, and
        inspect(L) + sptrsv, of each matrix)."""
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in D]
        stats = [[None, None] for _ in D]
        se = [torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)]
        se[0].record(stream)
        if args.streams == 1:
            for i, d in enumerate(D):
                one(d, stream, evs[i], record, stats, i)
        else:
            used = side if args.streams == 2 else side + side_l
            for s in used:
                s.wait_stream(stream)
            # host threads start one after another, each some 0.1-0.7 ms after
            # the last: the longest chains go first (the L chains, larger matrix
            # first, then the A chains)
            if args.streams == 2:
                jobs = [(one, i, side[i]) for i in order]
            else:
                jobs = [(chain_l, i, side_l[i]) for i in order] + [(chain_a, i, side[i]) for i in order]
            th = [threading.Thread(target=fn, args=(D[i], s, evs[i], record, stats, i)) for fn, i, s in jobs]
            for t in th:
                t.start()
            for t in th:
                t.join()
            for s in used:
                stream.wait_stream(s)
        se[1].record(stream)
        return evs, stats, se

    for _ in range(args.warmup):
        flush()
        step(False)
    torch.cuda.synchronize()
    serial = None
    if args.streams != 1:
        # the same steps with everything on one stream, for comparison (before
        # the timed steps, then the concurrent form is warmed up again)
        keep, args.streams = args.streams, 1
        step(False)
        sms = []
        for _ in range(args.steps):
            flush()
            sms.append(step(False)[2])
        torch.cuda.synchronize()
        args.streams = keep
        serial = float(np.mean([a.elapsed_time(b) for a, b in sms]))
        for _ in range(args.warmup):
            flush()
            step(False)
        torch.cuda.synchronize()
    launches0 = ddf.ddf_kernel_launches()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank)
    t0 = time.perf_counter()
    steps = []
    for _ in range(args.steps):
        flush()
        steps.append(step(False))
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    launches = ddf.ddf_kernel_launches() - launches0

    # per-phase times (ms) and bytes
    ph = {(d["name"], p): [] for d in D for p in phases}
    step_ms = []
    bounds = {"inspect_spmv": (0, 1), "spmv": (1, 2), "inspect_sptrsv": (3, 4), "sptrsv": (4, 5)}
    # timeline of the step: start and end of each chain after the step's start event
    tl = {(d["name"], c): [] for d in D for c in ("A", "L")}
    for evs, _, se in steps:
        for d, e in zip(D, evs):
            for p in phases:
                a, b = bounds[p]
                ph[(d["name"], p)].append(e[a].elapsed_time(e[b]))
            tl[(d["name"], "A")].append((se[0].elapsed_time(e[0]), se[0].elapsed_time(e[2])))
            tl[(d["name"], "L")].append((se[0].elapsed_time(e[3]), se[0].elapsed_time(e[5])))
        step_ms.append(se[0].elapsed_time(se[1]))
    timeline = {f"{nm}/{c}": [round(float(np.mean([t[0] for t in v])), 3), round(float(np.mean([t[1] for t in v])), 3)]
                for (nm, c), v in tl.items()}
    # plan statistics (a host copy of each plan), from one more step outside
    # the timed region; the plans are deterministic
    stats = step(True)[1]

    exec_b = sum(sa["bytes_exec"] + sl["bytes_exec"] for sa, sl in stats)
    ms, value = aggregate(float(np.mean(step_ms)), exec_b, world, dev)
    hbm, peak_kind = peaks()

    breakdown = {}
    for (d, (sa, sl)) in zip(D, stats):
        nm = d["name"]
        t_spmv = float(np.mean(ph[(nm, "spmv")]))
        t_trsv = float(np.mean(ph[(nm, "sptrsv")]))
        breakdown[nm] = {
            "inspect_spmv_ms": round(float(np.mean(ph[(nm, "inspect_spmv")])), 4),
            "spmv_ms": round(t_spmv, 4),
            "spmv_gbs": round(sa["bytes_exec"] / (t_spmv * 1e-3) / 1e9, 1),
            "spmv_bytes": sa["bytes_exec"],
            "inspect_sptrsv_ms": round(float(np.mean(ph[(nm, "inspect_sptrsv")])), 4),
            "sptrsv_ms": round(t_trsv, 4),
            "sptrsv_gbs": round(sl["bytes_exec"] / (t_trsv * 1e-3) / 1e9, 1),
            "sptrsv_bytes": sl["bytes_exec"],
            # FLOPs (Sec. V): SpMV 2 nnz; SpTRSV 2 (nnz_L - n) + n divisions
            "spmv_gflops": round(2 * sa["nnz"] / (t_spmv * 1e-3) / 1e9, 1),
            "sptrsv_gflops": round((2 * (sl["nnz"] - sl["n_rows"]) + sl["n_rows"]) / (t_trsv * 1e-3) / 1e9, 1),
            "depth": sl["levels"],
            "partitions": sl["depth"],
            "blocks": sl["blocks"],
            "codelets_spmv": sa["ncodelets"], "ops_spmv": sa["ops"],
            "codelets_sptrsv": sl["ncodelets"], "ops_sptrsv": sl["ops"],
        }
    # dominant executor call (by time) for the roofline object
    cand = []
    for nm, bd in breakdown.items():
        cand.append((bd["spmv_ms"], f"ddf_spmv[{nm}]", bd["spmv_bytes"]))
        cand.append((bd["sptrsv_ms"], f"ddf_sptrsv[{nm}]", bd["sptrsv_bytes"]))
    t_dom, dom, dom_bytes = max(cand)
    achieved = dom_bytes / (t_dom * 1e-3) / 1e9
    # DRAM bytes per launch: the ratio (dram read + write) / algorithmic bytes
    # from one ncu capture of the half-scale case, applied to this launch's
    # algorithmic bytes (the traffic scales with the rows processed).
    ratio = TRAFFIC_RATIO.get(dom)
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": hbm,
                "unit": "GB/s", "frac": round(achieved / hbm, 4),
                "traffic": round(ratio * dom_bytes) if ratio else None,
                "peak_source": f"{peak_kind} copy bandwidth"}

    critical = None if args.no_critical_path else critical_path(ddf, torch, dev, stream, breakdown, hbm)

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, D, ddf, torch, dev, stream, exec_b, world)
    mixed = None
    if not args.no_mixed:
        mixed = run_mixed(D, ddf, torch, stream, flush, breakdown)
    batched = None
    if not args.no_batch:
        del D
        torch.cuda.empty_cache()
        batched = run_batch(args, ddf, torch, dev, stream, flush)

    return {
        "value": value, "ms_per_step": ms, "wall_s": wall, "launches": launches, "clocks": clk,
        "breakdown": breakdown, "roofline": roofline, "critical_path": critical, "e2e": e2e,
        "serial_ms_per_step": serial, "timeline": timeline,
        "exec_bytes_per_step": exec_b,
        "mixed": mixed, "batched": batched,
    }


# (dram__bytes_read.sum + dram__bytes_write.sum) / algorithmic bytes of one
# launch, from one ncu capture of the half-scale workload (elasticity 32^3
# nodes: 38.59 MB of DRAM traffic for 36.34 MB of algorithmic bytes).
TRAFFIC_RATIO = {"ddf_sptrsv[elast3x3_64]": (38545152 + 47104) / 36341468}


def critical_path(ddf, torch, dev, stream, breakdown, hbm, n_chain=8192, reps=5):
    """The SpTRSV bound max(bytes / HBM bandwidth, depth x t_hop).  t_hop, the
    cost of one dependency level, is measured on a pure chain (a bidiagonal
    matrix: n levels of one row each) with the same executor."""
    ch = synth.chain(n_chain)
    td = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    q = ddf.ddf_inspect(td(ch.rowptr), td(ch.colidx), td(ch.values), ch.n_cols, ddf.DDF_SPTRSV)
    b = td(synth.uniform_vector(n_chain, 9))
    x = torch.empty(n_chain, dtype=torch.float64, device=dev)
    ts = []
    for i in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ddf.ddf_sptrsv(q, b, x, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        if i:
            ts.append(e0.elapsed_time(e1))
    if ddf.ddf_get_status(q, stream=stream) != 0:
        return None
    t_hop = float(np.median(ts)) * 1e3 / n_chain           # us per level
    out = {"t_hop_us": round(t_hop, 3), "chain_rows": n_chain}
    for nm, bd in breakdown.items():
        t_bw = bd["sptrsv_bytes"] / (hbm * 1e9) * 1e6           # us at the measured copy bandwidth
        t_lat = bd["depth"] * t_hop
        bound = max(t_bw, t_lat)
        meas = bd["sptrsv_ms"] * 1e3
        out[nm] = {"levels": bd["depth"], "bytes_bound_us": round(t_bw, 1), "depth_x_hop_us": round(t_lat, 1),
                   "bound": "latency" if t_lat >= t_bw else "hbm", "measured_us": round(meas, 1),
                   "frac_of_bound": round(bound / meas, 3)}
    return out


def run_batch(args, ddf, torch, dev, stream, flush, nrhs=32, reps=5):
    """The batching form: 256 uneven matrices (FP32 values), 32 right-hand
    sides each.  Batched: one block-diagonal plan per kind, tiles picked by
    ddf_tune, SpMM + SpTRSM recorded in one CUDA graph and replayed.  Compared
    with per-matrix launches of the same multi-RHS executors and with the
    plain path (the FP64 single-vector executors, one call per matrix and
    right-hand side)."""
    mats, rhs = synth.batch(args.batch_count, nrhs=nrhs)
    lows = [synth.lower_triangle(m) for m in mats]
    td = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    A = [(td(m.rowptr), td(m.colidx), td(m.values), m.n_cols) for m in mats]
    L = [(td(m.rowptr), td(m.colidx), td(m.values), m.n_cols) for m in lows]
    N = sum(m.n_rows for m in mats)
    X = td(np.concatenate(rhs))                     # [N][32] float32
    Y = torch.empty((N, nrhs), dtype=torch.float32, device=dev)
    Xs = torch.empty((N, nrhs), dtype=torch.float32, device=dev)
    o32 = ddf.ddf_opts_default(store_dtype=ddf.DDF_F32)
    pA = ddf.ddf_inspect_batch(A, ddf.DDF_SPMV, o32)
    pL = ddf.ddf_inspect_batch(L, ddf.DDF_SPTRSV, o32)
    tile_spmv = ddf.ddf_tune(pA, X, Y, nrhs)
    tile_trsv = ddf.ddf_tune(pL, X, Xs, nrhs)
    side = torch.cuda.Stream(device=dev)
    side.wait_stream(stream)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            ddf.ddf_spmm(pA, X, Y, nrhs, stream=side)
            ddf.ddf_sptrsm(pL, X, Xs, nrhs, stream=side)
    stream.wait_stream(side)

    def timed(fn, r=reps):
        ts = []
        for _ in range(r):
            flush()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    t_graph = timed(g.replay)
    st_graph = ddf.ddf_get_status(pL)
    sa, sl = ddf.ddf_plan_stats(pA), ddf.ddf_plan_stats(pL)
    nnzA, nnzL = sa["points"], sl["points"]
    # algorithmic bytes: FP32 values once, the 32-wide blocks read once and written once
    bytes_spmm = 4 * nnzA + 4 * nrhs * (sa["n_cols"] + sa["n_rows"]) + 4 * sa["ops"][2] + 64 * sum(sa["ncodelets"])
    bytes_trsm = 4 * nnzL + 4 * sl["n_rows"] + 4 * nrhs * 3 * sl["n_rows"] + 4 * sl["ops"][2] \
        + 64 * sum(sl["ncodelets"])
    # per-matrix launches of the same multi-RHS executors
    pa = [ddf.ddf_inspect(*a[:3], a[3], ddf.DDF_SPMV, o32) for a in A]
    pl = [ddf.ddf_inspect(*l[:3], l[3], ddf.DDF_SPTRSV, o32) for l in L]
    offs = np.concatenate([[0], np.cumsum([m.n_rows for m in mats])])

    def per_matrix():
        for i in range(len(mats)):
            a, b = int(offs[i]), int(offs[i + 1])
            ddf.ddf_spmm(pa[i], X[a:b], Y[a:b], nrhs)
            ddf.ddf_sptrsm(pl[i], X[a:b], Xs[a:b], nrhs)

    t_per = timed(per_matrix, 3)
    # the plain path: FP64 single-vector executors, one call per matrix and right-hand side
    pa64 = [ddf.ddf_inspect(*a[:3], a[3], ddf.DDF_SPMV) for a in A]
    pl64 = [ddf.ddf_inspect(*l[:3], l[3], ddf.DDF_SPTRSV) for l in L]
    X64 = X.double().t().contiguous()                # [32][N]
    Y64 = torch.empty_like(X64)
    S64 = torch.empty_like(X64)

    def plain():
        for i in range(len(mats)):
            a, b = int(offs[i]), int(offs[i + 1])
            for k in range(nrhs):
                ddf.ddf_spmv(pa64[i], X64[k, a:b], Y64[k, a:b])
                ddf.ddf_sptrsv(pl64[i], X64[k, a:b], S64[k, a:b])

    t_plain = timed(plain, 1)
    err = float(torch.linalg.norm(Y.double().t() - Y64) / torch.linalg.norm(Y64))
    errs = float(torch.linalg.norm(Xs.double().t() - S64) / torch.linalg.norm(S64))
    for p in pa + pl + pa64 + pl64 + [pA, pL]:
        p.destroy()
    return {"matrices": len(mats), "rows": int(N), "nnz": int(nnzA), "nnz_lower": int(nnzL), "nrhs": nrhs,
            "dtype": "f32 values and vectors, f32 sums", "tile_spmm_unit_nnz": tile_spmv,
            "tile_sptrsm_units_per_cta": tile_trsv, "graph_ms": round(t_graph, 4), "graph_status": st_graph,
            "graph_gbs": round((bytes_spmm + bytes_trsm) / (t_graph * 1e-3) / 1e9, 1),
            "per_matrix_multi_rhs_ms": round(t_per, 3), "speedup_vs_per_matrix": round(t_per / t_graph, 2),
            "plain_fp64_per_rhs_ms": round(t_plain, 2), "speedup_vs_plain_fp64": round(t_plain / t_graph, 2),
            "spmm_relerr_vs_fp64": err, "sptrsm_relerr_vs_fp64": errs}


def run_mixed(D, ddf, torch, stream, flush, breakdown, reps=5):
    """FP32 / BF16 executors against the FP64 ones on the same matrices: SpMV
    with low-precision values and vectors (FP32 sums), SpTRSV as low-precision
    solves refined in FP64 to a relative residual of 1e-12.  Errors are stated
    against the FP64 executor's result (itself within 1e-12 of the FP64 CPU
    oracle in the parity tests)."""
    out = {}

    def timed(fn):
        ts = []
        for _ in range(reps):
            flush()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    for d in D:
        nm = d["name"]
        a, lo = d["a"], d["lo"]
        res = {}
        p64 = ddf.ddf_inspect(*d["A"], a.n_cols, ddf.DDF_SPMV)
        ddf.ddf_spmv(p64, d["x"], d["y"])
        y64 = d["y"].clone()
        t64 = timed(lambda: ddf.ddf_spmv(p64, d["x"], d["y"]))
        st64 = ddf.ddf_plan_stats(p64)
        res["spmv_f64_ms"] = round(t64, 4)
        for dt, tdt, name, vs in ((ddf.DDF_F32, torch.float32, "f32", 4), (ddf.DDF_BF16, torch.bfloat16, "bf16", 2)):
            pl = ddf.ddf_inspect(*d["A"], a.n_cols, ddf.DDF_SPMV, ddf.ddf_opts_default(store_dtype=dt))
            xl = d["x"].to(tdt)
            yl = torch.empty(a.n_rows, dtype=tdt, device=d["x"].device)
            t = timed(lambda: ddf.ddf_spmv_lowp(pl, xl, yl))
            err = float(torch.linalg.norm(yl.double() - y64) / torch.linalg.norm(y64))
            lp_bytes = st64["bytes_exec"] - (8 - vs) * (st64["points"] + a.n_cols + a.n_rows)
            res[f"spmv_{name}_ms"] = round(t, 4)
            res[f"spmv_{name}_speedup"] = round(t64 / t, 3)
            res[f"spmv_{name}_gbs"] = round(lp_bytes / (t * 1e-3) / 1e9, 1)
            res[f"spmv_{name}_relerr"] = err
            pl.destroy()
        p64.destroy()
        q64 = ddf.ddf_inspect(*d["L"], lo.n_cols, ddf.DDF_SPTRSV)
        ddf.ddf_sptrsv(q64, d["b"], d["xs"])
        x64 = d["xs"].clone()
        tq = timed(lambda: ddf.ddf_sptrsv(q64, d["b"], d["xs"]))
        res["sptrsv_f64_ms"] = round(tq, 4)
        q64.destroy()
        for dt, name in ((ddf.DDF_F32, "f32"), (ddf.DDF_BF16, "bf16")):
            ql = ddf.ddf_inspect(*d["L"], lo.n_cols, ddf.DDF_SPTRSV, ddf.ddf_opts_default(store_dtype=dt))
            xr = torch.empty(lo.n_rows, dtype=torch.float64, device=d["x"].device)
            info = {}

            def go():
                info["r"] = ddf.ddf_sptrsv_refine(ql, d["b"], xr, tol=1e-12, max_iter=30)

            t = timed(go)
            st, iters, rel = info["r"]
            res[f"sptrsv_refine_{name}_ms"] = round(t, 4)
            res[f"sptrsv_refine_{name}_speedup"] = round(tq / t, 3)
            res[f"sptrsv_refine_{name}_iters"] = iters
            res[f"sptrsv_refine_{name}_relres"] = rel
            res[f"sptrsv_refine_{name}_status"] = st
            res[f"sptrsv_refine_{name}_relerr"] = float(torch.linalg.norm(xr - x64) / torch.linalg.norm(x64))
            ql.destroy()
        out[nm] = res
    return out


def run_e2e(args, D, ddf, torch, dev, stream, exec_b, world):
    """Same step from pinned host buffers: CSR, x and b copied in, y and x read back."""
    H = []
    h2d = d2h = 0
    for d in D:
        a, lo = d["a"], d["lo"]
        pin = lambda v: torch.from_numpy(np.ascontiguousarray(v)).pin_memory()  # noqa: E731
        H.append({"A": (pin(a.rowptr), pin(a.colidx), pin(a.values)),
                  "L": (pin(lo.rowptr), pin(lo.colidx), pin(lo.values)),
                  "x": pin(d["x"].cpu().numpy()), "b": pin(d["b"].cpu().numpy()),
                  "y": torch.empty(a.n_rows, dtype=torch.float64).pin_memory(),
                  "xs": torch.empty(lo.n_rows, dtype=torch.float64).pin_memory()})
        h2d += csr_bytes(a) + csr_bytes(lo) + 8 * a.n_cols + 8 * lo.n_rows
        d2h += 8 * a.n_rows + 8 * lo.n_rows

    # The four chains (inspect(A) + spmv and inspect(L) + sptrsv of each
    # matrix) run on their own streams and host threads, as in the
    # device-resident step.  Uploads go on one copy stream, longest chain
    # first (the L chains, larger matrix first, then the A chains), and each
    # chain's stream waits only for its own arrays: the long solve chains
    # start while the remaining arrays are still being copied, instead of
    # after all of them.
    opts_L = ddf.ddf_opts_default(coarsen_rows=args.coarsen) if args.coarsen is not None else None
    copy = torch.cuda.Stream(device=dev)
    size = lambda i: D[i]["a"].nnz + D[i]["lo"].nnz  # noqa: E731
    by_size = sorted(range(len(D)), key=lambda i: -size(i))
    order = [("L", i) for i in by_size] + [("A", i) for i in by_size]
    lo_p, hi_p = torch.cuda.Stream.priority_range() if hasattr(torch.cuda.Stream, "priority_range") else (0, -1)
    streams = {job: torch.cuda.Stream(device=dev, priority=hi_p if job[1] == by_size[0] else lo_p)
               for job in order}

    def upload(arrs):
        return tuple(t.to(dev, non_blocking=True) for t in arrs)

    def run(kind, i, g, ev):
        torch.cuda.set_device(dev)
        s, d, h = streams[(kind, i)], D[i], H[i]
        s.wait_event(ev)
        for t in g:
            t.record_stream(s)
        with torch.cuda.stream(s):
            if kind == "A":
                p = ddf.ddf_inspect(*g[:3], d["a"].n_cols, ddf.DDF_SPMV, None, s)
                out = torch.empty(d["a"].n_rows, dtype=torch.float64, device=dev)
                ddf.ddf_spmv(p, g[3], out, stream=s)
                h["y"].copy_(out, non_blocking=True)
            else:
                p = ddf.ddf_inspect(*g[:3], d["lo"].n_cols, ddf.DDF_SPTRSV, opts_L, s)
                out = torch.empty(d["lo"].n_rows, dtype=torch.float64, device=dev)
                ddf.ddf_sptrsv(p, g[3], out, stream=s)
                h["xs"].copy_(out, non_blocking=True)
            p.destroy()

    def step():
        copy.wait_stream(stream)
        for s in streams.values():
            s.wait_stream(stream)
        jobs = []
        with torch.cuda.stream(copy):
            for kind, i in order:
                h = H[i]
                g = upload(h["A"]) + (h["x"].to(dev, non_blocking=True),) if kind == "A" else \
                    upload(h["L"]) + (h["b"].to(dev, non_blocking=True),)
                ev = torch.cuda.Event()
                ev.record(copy)
                jobs.append((kind, i, g, ev))
        th = [threading.Thread(target=run, args=job) for job in jobs]
        for t in th:
            t.start()
        for t in th:
            t.join()
        for s in streams.values():
            stream.wait_stream(s)
        stream.wait_stream(copy)

    for _ in range(max(1, args.warmup)):
        step()
    torch.cuda.synchronize()
    times = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    ms, v = aggregate(float(np.mean(times)), exec_b, world, dev)
    return {"value": round(v, 2), "unit": "GB/s",
            "ms_per_step": round(ms, 3), "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}


# ---------------------------------------------------------------------------
# the oracle on the host cores (CPU baseline and reference arm)
# ---------------------------------------------------------------------------
def oracle_step(mats):
    import oracle
    for name, a, lo, x, b in mats:
        oracle.inspect(a, oracle.SPMV)
        oracle.spmv(a, x)
        oracle.inspect(lo, oracle.SPTRSV)
        oracle.sptrsv(lo, b)


def oracle_exec_bytes(mats):
    """Executor algorithmic bytes of the oracle's plans, counted like the
    library's plan statistics."""
    import oracle
    total = 0
    for name, a, lo, x, b in mats:
        for kind, m in ((oracle.SPMV, a), (oracle.SPTRSV, lo)):
            p = oracle.inspect(m, kind)
            r = p.records
            lens = np.diff(m.rowptr.astype(np.int64))[p.perm] - (1 if kind == oracle.SPTRSV else 0)
            cs = np.concatenate([[0], np.cumsum(lens)])
            ops2 = sum(int(cs[q + mm] - cs[q]) for q, mm in zip(r[r[:, 1] == 2][:, 2], r[r[:, 1] == 2][:, 3]))
            idx_rows = int((r[r[:, 1] == 2][:, 3] + 1).sum())
            sent = int(r[r[:, 1] == 1][:, 4].sum())
            perm_rows = int(r[r[:, 5] == 0][:, 3].sum())
            pts = int(lens.sum())
            n = m.n_rows
            if kind == oracle.SPMV:
                total += 8 * pts + 8 * m.n_cols + 8 * n + 4 * ops2 + 4 * idx_rows + 4 * sent + 64 * len(r)
            else:
                total += 8 * pts + 32 * n + 4 * ops2 + 4 * idx_rows + 4 * perm_rows + 4 * sent + 64 * len(r)
    return total


def run_oracle(mats, seconds, max_steps=None, warmup=0):
    import oracle
    oracle.build()
    for _ in range(warmup):
        oracle_step(mats)
    times = []
    t_end = time.perf_counter() + seconds
    while True:
        t0 = time.perf_counter()
        oracle_step(mats)
        times.append(time.perf_counter() - t0)
        if max_steps is not None and len(times) >= max_steps:
            break
        if max_steps is None and time.perf_counter() > t_end:
            break
    return times


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return 0
        mats = build_inputs(args.scale)
        times = run_oracle(mats, 0, max_steps=args.steps, warmup=args.warmup)
        b = oracle_exec_bytes(mats)
        ms = 1e3 * float(np.mean(times))
        v = b / (ms * 1e-3) / 1e9
        line = {"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "GB/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(ms, 2), "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": "+".join(WORKLOAD), "scale": args.scale},
                "cpu_baseline": {"value": round(v, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
                                 "sample": "the full workload per step, sequential C oracle"},
                "e2e": {"value": round(v, 4), "unit": "GB/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0

    import torch
    if world > 1:
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        torch.distributed.init_process_group(backend=backend)
    r = run_ours(args, rank, world, local_rank)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        mats = build_inputs(args.scale)
        times = run_oracle(mats, args.cpu_seconds)
        b = oracle_exec_bytes(mats)
        cv = b / float(np.mean(times)) / 1e9
        cpu = {"value": round(cv, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
               "sample": f"{len(times)} full steps of the workload (sequential C oracle, "
                         f"{sum(times):.1f} s)", "exec_bytes_oracle_plan": b}
    if rank == 0:
        hbm, _ = peaks()
        line = {
            "metric": METRIC, "value": round(r["value"], 2), "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(r["ms_per_step"], 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "+".join(WORKLOAD), "scale": args.scale,
                       "step": "inspect(A)+spmv+inspect(L)+sptrsv per matrix",
                       "l2": "256 MB written then another 256 MB read between steps (the flush's "
                             "write-back happens before the timed work); inputs larger than L2",
                       "streams": {1: "everything on one stream",
                                   2: "one stream and host thread per matrix",
                                   4: "one stream and host thread per chain: inspect(A)+spmv, "
                                      "inspect(L)+sptrsv of each matrix"}[args.streams],
                       "parallelism": "replicas" if world > 1 else "single"},
            "frac_of_hbm": round(r["value"] / hbm, 4),
            "roofline": r["roofline"],
            "critical_path": r["critical_path"],
            "serial": None if r["serial_ms_per_step"] is None else {
                "ms_per_step": round(r["serial_ms_per_step"], 4),
                "value": round(r["exec_bytes_per_step"] / (r["serial_ms_per_step"] * 1e-3) / 1e9, 2)},
            "cpu_baseline": cpu,
            "e2e": r["e2e"],
            "gpu_launches": r["launches"],
            "clocks": r["clocks"],
            "breakdown": r["breakdown"],
            # [start, end] of each chain (A: inspect(A) + spmv, L: inspect(L) +
            # sptrsv) in ms after the step's start event, mean over the timed steps
            "timeline_ms": r["timeline"],
            "mixed_precision": r["mixed"],
            "batched": r["batched"],
            "exec_bytes_per_step": r["exec_bytes_per_step"],
        }
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
