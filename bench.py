#!/usr/bin/env python
"""Benchmark of the DDF hot path on one GB300 (or N independent replicas).

One step = the whole path over the headline workload (default "st27_168": a
3-D 27-point stencil on a 168^3 grid, 4.74M rows, 126.5M nonzeros, the
largest single-GPU configuration): for each matrix A and its lower triangle L,
    ddf_inspect(A, SpMV) -> ddf_spmv      ddf_inspect(L, SpTRSV) -> ddf_sptrsv
with CSR inputs and vectors already resident in HBM.  ``value`` is the
executors' algorithmic bytes (plan statistics) moved per second of the whole
step, inspection included.  Extra keys report:
  exec_only        the executors alone with their plans reused (Sec. V-C amortisation)
  roofline         the dominant executor call of the step against the measured HBM copy bandwidth
  roofline_spmv    the SpMV alone, with its FP64-pipe ceiling
  critical_path    the SpTRSV bound max(bytes / bandwidth, depth x t_hop)
  extra            other workloads (default the power-law matrix), each phase alone
  mixed_precision  FP32 / BF16 SpMV and refined SpTRSV on the 27-point stencil, integer
                   and N(0,1) values, errors against the CPU oracle
  ablation_e5      plans restricted to BLAS + PSC II codelets against all types (Sec. V); Eq. 1's
                   weights recalibrated on the GPU (ddf_tune_cost)
  blas_banded      a band matrix, whose plan is BLAS codelets
  batched          256 uneven matrices x 32 right-hand sides in one CUDA graph

``--impl reference`` times the CPU oracle (plain sequential C, FP64) on the
host cores over the same workload and prints the same line with
``"impl": "reference"``.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "SpMV & SpTRSV GB/s as % of HBM roofline; mixed-precision vs FP64 speedup"
DEFAULT_WORKLOAD = "st27_168"
DEFAULT_EXTRA = "powerlaw_4m"
DEFAULT_MIXED = "st27_168+st27r_168"
DEFAULT_ABLATION = "st27_168+lap7_128"
L2_FLUSH_BYTES = 256 << 20
FALLBACK_HBM_GBS = 6800.0
# FP64 fused multiply-adds one GB300 SM issues per clock (1.25 TFLOP/s nominal
# FP64 over 152 SMs at 2.07 GHz): one per stored value of an FP64 SpMV, which
# caps it below the HBM bandwidth
FP64_FMA_PER_SM_CLK = 2


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD,
                    help="matrices of the timed step, joined by '+' (names of synth.WORKLOADS)")
    ap.add_argument("--extra", default=DEFAULT_EXTRA, help="workloads timed phase by phase ('' = none)")
    ap.add_argument("--mixed", default=DEFAULT_MIXED, help="workloads of the mixed-precision section")
    ap.add_argument("--ablation", default=DEFAULT_ABLATION, help="workloads of the E5 ablation")
    ap.add_argument("--scale", type=float, default=1.0, help="grid scale (1.0 = the full workload)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-ablation", action="store_true")
    ap.add_argument("--no-banded", action="store_true")
    ap.add_argument("--no-critical-path", action="store_true", help="skip the chain solve that measures t_hop")
    ap.add_argument("--streams", type=int, default=4, choices=[1, 2, 4],
                    help="1: everything on one stream; 2: one stream and host thread per matrix; "
                         "4 (default): one per chain, inspect(A)+spmv and inspect(L)+sptrsv of each matrix")
    ap.add_argument("--serial", action="store_true", help="same as --streams 1")
    ap.add_argument("--prio", default="chain", choices=["chain", "size", "achain"],
                    help="stream priorities: 'chain' (default) gives the inspect(L) + sptrsv chains the high "
                         "priority and the inspect(A) + spmv chains the low one; 'achain' the reverse; 'size' "
                         "gives both chains of the largest matrix the high priority")
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--coarsen", type=int, default=None,
                    help="SpTRSV rows per block (coarsen_rows; 0 = plain level sets; default: library default)")
    a = ap.parse_args(argv)
    if a.serial:
        a.streams = 1
    return a


def names(spec):
    return [s for s in (spec or "").split("+") if s]


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def build_inputs(workload, scale):
    mats = []
    for name in names(workload):
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

    def __init__(self, gpu_index, interval_ms=100):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", str(interval_ms)],
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
        names_ = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names_[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
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


def make_timer(torch, stream, flush):
    def timed(fn, reps=5):
        """Median device time (ms) of fn over `reps` calls, L2 flushed before each."""
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
    return timed


def sptrsv_flops(st):
    # Sec. V: SpTRSV = 2 (nnz_L - n) + n divisions
    return 2 * (st["nnz"] - st["n_rows"]) + st["n_rows"]


def solo(ddf, torch, dev, timed, a, lo, x, b, opts_a=None, opts_l=None, do_sptrsv=True):
    """Each phase of one matrix alone on the GPU: inspection of A and L, then
    the SpMV and the SpTRSV with their plans reused.  Median of 5, L2 flushed."""
    td = lambda v: torch.from_numpy(np.ascontiguousarray(v)).to(dev)  # noqa: E731
    A = (td(a.rowptr), td(a.colidx), td(a.values))
    xd = td(x)
    y = torch.empty(a.n_rows, dtype=torch.float64, device=dev)
    out = {"n": a.n_rows, "nnz": a.nnz}
    holder = {}

    def insp_a():
        if "pA" in holder:
            holder.pop("pA").destroy()
        holder["pA"] = ddf.ddf_inspect(*A, a.n_cols, ddf.DDF_SPMV, opts_a)
    out["inspect_spmv_ms"] = round(timed(insp_a), 4)
    pA = holder.pop("pA")
    sa = ddf.ddf_plan_stats(pA)
    t = timed(lambda: ddf.ddf_spmv(pA, xd, y))
    out.update({"spmv_ms": round(t, 4), "spmv_bytes": sa["bytes_exec"],
                "spmv_gbs": round(sa["bytes_exec"] / (t * 1e-3) / 1e9, 1),
                "spmv_gflops": round(2 * sa["nnz"] / (t * 1e-3) / 1e9, 1),
                "codelets_spmv": sa["ncodelets"], "ops_spmv": sa["ops"], "units_spmv": sa["nunits"]})
    pA.destroy()
    del A
    if do_sptrsv:
        L = (td(lo.rowptr), td(lo.colidx), td(lo.values))
        bd = td(b)
        xs = torch.empty(lo.n_rows, dtype=torch.float64, device=dev)

        def insp_l():
            if "pL" in holder:
                holder.pop("pL").destroy()
            holder["pL"] = ddf.ddf_inspect(*L, lo.n_cols, ddf.DDF_SPTRSV, opts_l)
        out["inspect_sptrsv_ms"] = round(timed(insp_l), 4)
        pL = holder.pop("pL")
        sl = ddf.ddf_plan_stats(pL)
        t = timed(lambda: ddf.ddf_sptrsv(pL, bd, xs))
        out.update({"sptrsv_ms": round(t, 4), "sptrsv_bytes": sl["bytes_exec"],
                    "sptrsv_gbs": round(sl["bytes_exec"] / (t * 1e-3) / 1e9, 1),
                    "sptrsv_gflops": round(sptrsv_flops(sl) / (t * 1e-3) / 1e9, 1),
                    "sptrsv_status": ddf.ddf_get_status(pL), "depth": sl["levels"],
                    "codelets_sptrsv": sl["ncodelets"], "ops_sptrsv": sl["ops"]})
        pL.destroy()
    return out


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_2111_12243_gb300 as ddf
    from paper_2111_12243_gb300 import build as ddf_build

    ddf_build.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    mats = build_inputs(args.workload, args.scale)

    def to_dev(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    D = []
    for name, a, lo, x, b in mats:
        D.append({
            "name": name, "a": a, "lo": lo, "xh": x, "bh": b,
            "A": (to_dev(a.rowptr), to_dev(a.colidx), to_dev(a.values)),
            "L": (to_dev(lo.rowptr), to_dev(lo.colidx), to_dev(lo.values)),
            "x": to_dev(x), "b": to_dev(b),
            "y": torch.empty(a.n_rows, dtype=torch.float64, device=dev),
            "xs": torch.empty(lo.n_rows, dtype=torch.float64, device=dev),
        })
    flush = L2Flush(torch, dev)
    timed = make_timer(torch, stream, flush)
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

    # The inspect(L) + sptrsv chains are the longer, latency-bound pipelines:
    # by default their streams get the higher priority and the bandwidth-bound
    # inspect(A) + spmv chains fill the SMs they leave idle ('--prio size':
    # both chains of the largest matrix high, the others low).
    order = sorted(range(len(D)), key=lambda i: -(D[i]["a"].nnz + D[i]["lo"].nnz))
    lo_p, hi_p = torch.cuda.Stream.priority_range() if hasattr(torch.cuda.Stream, "priority_range") else (0, -1)
    if args.prio == "chain":
        prio_a = {i: lo_p for i in range(len(D))}
        prio_l = {i: hi_p for i in range(len(D))}
    elif args.prio == "achain":
        prio_a = {i: hi_p for i in range(len(D))}
        prio_l = {i: lo_p for i in range(len(D))}
    else:
        prio_a = prio_l = {i: (hi_p if k == 0 else lo_p) for k, i in enumerate(order)}
    side = [torch.cuda.Stream(device=dev, priority=prio_a[i]) for i in range(len(D))]
    side_l = [torch.cuda.Stream(device=dev, priority=prio_l[i]) for i in range(len(D))]

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
            # host threads start one after another: the longest chains go
            # first (the L chains, larger matrix first, then the A chains)
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

    # clocks are sampled from the first warm-up step until the executors have
    # also been timed alone (a window of seconds, the timed steps inside it)
    clocks = ClockSampler(local_rank)
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
    t0 = time.perf_counter()
    steps = []
    for _ in range(args.steps):
        flush()
        steps.append(step(False))
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    if world > 1:
        torch.distributed.barrier()
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
            "sptrsv_gflops": round(sptrsv_flops(sl) / (t_trsv * 1e-3) / 1e9, 1),
            "nnz": sa["nnz"], "nnz_lower": sl["nnz"],
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
    # from one ncu capture of a smaller case of the same kernel, applied to
    # this launch's algorithmic bytes (the traffic scales with the rows).
    ratio = TRAFFIC_RATIO.get(dom)
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": hbm,
                "unit": "GB/s", "frac": round(achieved / hbm, 4),
                "traffic": round(ratio * dom_bytes) if ratio else None,
                "peak_source": f"{peak_kind} copy bandwidth",
                "timed": "CUDA events around the call on its stream, inside the timed steps"}

    # the executors alone, their plans reused (the amortised case of Sec. V-C)
    exec_only = {}
    for d in D:
        exec_only[d["name"]] = solo(ddf, torch, dev, timed, d["a"], d["lo"], d["xh"], d["bh"], None, opts_L)
    clk = clocks.stop()
    clk["window"] = "warm-up steps, timed steps and the executors alone"
    # SpMV of the first matrix: roofline against HBM and its FP64-pipe ceiling
    e0 = exec_only[D[0]["name"]]
    f_clk = (clk.get("sm_mhz") or 2070.0) * 1e6
    ceil = e0["spmv_bytes"] * FP64_FMA_PER_SM_CLK * n_sm * f_clk / e0["nnz"] / 1e9
    roofline_spmv = {"bound": "hbm", "kernel": f"ddf_spmv[{D[0]['name']}]", "achieved": e0["spmv_gbs"],
                     "peak": hbm, "unit": "GB/s", "frac": round(e0["spmv_gbs"] / hbm, 4),
                     "traffic": round(TRAFFIC_RATIO[f"ddf_spmv[{D[0]['name']}]"] * e0["spmv_bytes"])
                     if f"ddf_spmv[{D[0]['name']}]" in TRAFFIC_RATIO else None,
                     "fp64_fma_ceiling_gbs": round(ceil, 1),
                     "frac_of_fp64_ceiling": round(e0["spmv_gbs"] / ceil, 4),
                     "fp64_ceiling": f"{FP64_FMA_PER_SM_CLK} FP64 FMA per SM per clock x {n_sm} SMs x "
                                     f"{f_clk / 1e6:.0f} MHz, one FMA per nonzero, "
                                     f"{e0['spmv_bytes'] / e0['nnz']:.2f} algorithmic bytes per nonzero",
                     "timed": "alone, median of 5, L2 flushed"}

    t_hop = None if args.no_critical_path else chain_hop(ddf, torch, dev, stream)
    critical = None if t_hop is None else critical_path(t_hop, breakdown, exec_only, hbm)

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, D, ddf, torch, dev, stream, exec_b, world)
    host = {d["name"]: (d["a"], d["lo"], d["xh"], d["bh"]) for d in D}
    del D
    torch.cuda.empty_cache()
    extra = None
    if names(args.extra):
        extra = {}
        for nm in names(args.extra):
            a, lo, x, b = synth.workload(nm, args.scale)
            r = solo(ddf, torch, dev, timed, a, lo, x, b, None, opts_L)
            if t_hop is not None:
                t_bw = r["sptrsv_bytes"] / (hbm * 1e9) * 1e6
                t_lat = r["depth"] * t_hop
                r["critical_path"] = {"levels": r["depth"], "bytes_bound_us": round(t_bw, 1),
                                      "depth_x_hop_us": round(t_lat, 1),
                                      "bound": "latency" if t_lat >= t_bw else "hbm",
                                      "measured_us": round(r["sptrsv_ms"] * 1e3, 1),
                                      "us_per_level": round(r["sptrsv_ms"] * 1e3 / max(r["depth"], 1), 3),
                                      "frac_of_bound": round(max(t_bw, t_lat) / (r["sptrsv_ms"] * 1e3), 3)}
            r["spmv_frac_of_hbm"] = round(r["spmv_gbs"] / hbm, 4)
            extra[nm] = r
            del a, lo
    mixed = None
    if not args.no_mixed and names(args.mixed):
        mixed = run_mixed(args, host, ddf, torch, dev, timed)
    ablation = None
    if not args.no_ablation and names(args.ablation):
        ablation = run_ablation(args, host, ddf, torch, dev, timed)
    banded = None
    if not args.no_banded:
        banded = run_banded(args, ddf, torch, dev, timed, hbm)
    batched = None
    if not args.no_batch:
        torch.cuda.empty_cache()
        batched = run_batch(args, ddf, torch, dev, stream, flush)

    return {
        "value": value, "ms_per_step": ms, "wall_s": wall, "launches": launches, "clocks": clk,
        "breakdown": breakdown, "roofline": roofline, "roofline_spmv": roofline_spmv,
        "critical_path": critical, "e2e": e2e, "exec_only": exec_only,
        "serial_ms_per_step": serial, "timeline": timeline,
        "exec_bytes_per_step": exec_b, "extra": extra,
        "mixed": mixed, "ablation": ablation, "banded": banded, "batched": batched,
    }


# (dram__bytes_read.sum + dram__bytes_write.sum) / algorithmic bytes of one
# call, from one ncu capture of a smaller case of the same kernels (the
# 27-point stencil at 126^3; the captures are summarised under profiles/).
# The traffic grows with the rows processed, so the ratio carries over.
TRAFFIC_RATIO = {
    "ddf_sptrsv[st27_168]": (297527552 + 14641664) / 280366928,
    "ddf_spmv[st27_168]": (460305152 + 4723456) / 463476904,
}


def chain_hop(ddf, torch, dev, stream, n_chain=8192, reps=5):
    """t_hop, the cost of one dependency level (us), measured on a pure chain
    (a bidiagonal matrix: n levels of one row each) with the same executor."""
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
    ok = ddf.ddf_get_status(q, stream=stream) == 0
    q.destroy()
    return float(np.median(ts)) * 1e3 / n_chain if ok else None


def critical_path(t_hop, breakdown, exec_only, hbm, n_chain=8192):
    """The SpTRSV bound max(bytes / HBM bandwidth, depth x t_hop), against the
    solve inside the step and alone."""
    out = {"t_hop_us": round(t_hop, 3), "chain_rows": n_chain}
    for nm, bd in breakdown.items():
        t_bw = bd["sptrsv_bytes"] / (hbm * 1e9) * 1e6           # us at the measured copy bandwidth
        t_lat = bd["depth"] * t_hop
        bound = max(t_bw, t_lat)
        meas = bd["sptrsv_ms"] * 1e3
        alone = exec_only[nm]["sptrsv_ms"] * 1e3
        out[nm] = {"levels": bd["depth"], "bytes_bound_us": round(t_bw, 1), "depth_x_hop_us": round(t_lat, 1),
                   "bound": "latency" if t_lat >= t_bw else "hbm", "measured_us": round(meas, 1),
                   "frac_of_bound": round(bound / meas, 3), "alone_us": round(alone, 1),
                   "alone_us_per_level": round(alone / max(bd["depth"], 1), 3),
                   "alone_frac_of_bound": round(bound / alone, 3)}
    return out


def run_batch(args, ddf, torch, dev, stream, flush, nrhs=32, reps=5):
    """The batching form: 256 uneven matrices (FP32 values), 32 right-hand
    sides each.  Batched: one block-diagonal plan per kind, work shapes picked
    by ddf_tune, the SpMV and the SpTRSV of the whole batch in one launch
    (ddf_batch_run, after the solve's fill) recorded in a CUDA graph and
    replayed.  Compared with the same two executors as separate calls (also
    in a graph), with per-matrix launches of them, and with the plain path
    (the FP64 single-vector executors, one call per matrix and right-hand
    side)."""
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
    g = torch.cuda.CUDAGraph()           # one launch for both executors
    g2 = torch.cuda.CUDAGraph()          # the two executors as separate calls
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            ddf.ddf_batch_run(pA, X, Y, pL, X, Xs, nrhs, stream=side)
        launches_one = ddf.ddf_last_launches(pL) + ddf.ddf_last_launches(pA)
        with torch.cuda.graph(g2, stream=side):
            ddf.ddf_spmm(pA, X, Y, nrhs, stream=side)
            ddf.ddf_sptrsm(pL, X, Xs, nrhs, stream=side)
        launches_two = ddf.ddf_last_launches(pL) + ddf.ddf_last_launches(pA)
    stream.wait_stream(side)
    timed = make_timer(torch, stream, flush)

    t_graph = timed(g.replay, reps)
    st_graph = ddf.ddf_get_status(pL)
    t_graph2 = timed(g2.replay, reps)
    t_spmm = timed(lambda: ddf.ddf_spmm(pA, X, Y, nrhs), reps)
    t_trsm = timed(lambda: ddf.ddf_sptrsm(pL, X, Xs, nrhs), reps)
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
    g.replay()
    torch.cuda.synchronize()
    err = float(torch.linalg.norm(Y.double().t() - Y64) / torch.linalg.norm(Y64))
    errs = float(torch.linalg.norm(Xs.double().t() - S64) / torch.linalg.norm(S64))
    for p in pa + pl + pa64 + pl64 + [pA, pL]:
        p.destroy()
    return {"matrices": len(mats), "rows": int(N), "nnz": int(nnzA), "nnz_lower": int(nnzL), "nrhs": nrhs,
            "sptrsm_levels": sl["levels"],
            "sptrsm_us_per_level": round(t_trsm * 1e3 / max(sl["levels"], 1), 3),
            "dtype": "f32 values and vectors, f32 sums", "tile_spmm_unit_nnz": tile_spmv,
            "tile_sptrsm_units_per_ticket": tile_trsv, "graph_ms": round(t_graph, 4), "graph_status": st_graph,
            "graph_gbs": round((bytes_spmm + bytes_trsm) / (t_graph * 1e-3) / 1e9, 1),
            "graph_launches": launches_one, "graph_two_calls_ms": round(t_graph2, 4),
            "graph_two_calls_gbs": round((bytes_spmm + bytes_trsm) / (t_graph2 * 1e-3) / 1e9, 1),
            "graph_two_calls_launches": launches_two,
            "spmm_ms": round(t_spmm, 4), "spmm_gbs": round(bytes_spmm / (t_spmm * 1e-3) / 1e9, 1),
            "sptrsm_ms": round(t_trsm, 4), "sptrsm_gbs": round(bytes_trsm / (t_trsm * 1e-3) / 1e9, 1),
            "per_matrix_multi_rhs_ms": round(t_per, 3), "speedup_vs_per_matrix": round(t_per / t_graph, 2),
            "plain_fp64_per_rhs_ms": round(t_plain, 2), "speedup_vs_plain_fp64": round(t_plain / t_graph, 2),
            "spmm_relerr_vs_fp64": err, "sptrsm_relerr_vs_fp64": errs}


def relerr(a, b):
    nb = float(np.linalg.norm(b))
    return float(np.linalg.norm(np.asarray(a, dtype=np.float64) - b) / nb) if nb > 0 else float(
        np.linalg.norm(np.asarray(a, dtype=np.float64) - b))


def run_mixed(args, host, ddf, torch, dev, timed):
    """The precision form: FP32 / BF16 executors against the FP64 ones on the
    same matrices.  SpMV with low-precision values and vectors (FP32 sums);
    SpTRSV as low-precision solves refined in FP64 to a relative residual of
    1e-12.  Errors are stated against the CPU oracle's FP64 results, which the
    CPU-baseline leg computes (oracle_references); without that leg they are
    stated against the GPU FP64 executors."""
    refs = None if args.no_cpu_baseline else oracle_references(args, host)
    out = {}
    td = lambda v: torch.from_numpy(np.ascontiguousarray(v)).to(dev)  # noqa: E731
    for nm in names(args.mixed):
        a, lo, x, b = host[nm] if nm in host else synth.workload(nm, args.scale)
        A = (td(a.rowptr), td(a.colidx), td(a.values))
        L = (td(lo.rowptr), td(lo.colidx), td(lo.values))
        xd, bd = td(x), td(b)
        y = torch.empty(a.n_rows, dtype=torch.float64, device=dev)
        xs = torch.empty(lo.n_rows, dtype=torch.float64, device=dev)
        res = {"values": "integer 26 / -1" if nm.startswith("st27_") else "N(0,1), diagonal 1 + sum |row|"}
        p64 = ddf.ddf_inspect(*A, a.n_cols, ddf.DDF_SPMV)
        t64 = timed(lambda: ddf.ddf_spmv(p64, xd, y))
        y64 = y.cpu().numpy()
        st64 = ddf.ddf_plan_stats(p64)
        p64.destroy()
        ref_y = refs[nm]["y"] if refs else y64
        res["against"] = "cpu oracle (fp64)" if refs else "gpu fp64 executor"
        res["spmv_f64_ms"] = round(t64, 4)
        res["spmv_f64_gbs"] = round(st64["bytes_exec"] / (t64 * 1e-3) / 1e9, 1)
        res["spmv_f64_relerr"] = relerr(y64, ref_y)
        for dt, tdt, name, vs in ((ddf.DDF_F32, torch.float32, "f32", 4), (ddf.DDF_BF16, torch.bfloat16, "bf16", 2)):
            pl = ddf.ddf_inspect(*A, a.n_cols, ddf.DDF_SPMV, ddf.ddf_opts_default(store_dtype=dt))
            xl = xd.to(tdt)
            yl = torch.empty(a.n_rows, dtype=tdt, device=dev)
            t = timed(lambda: ddf.ddf_spmv_lowp(pl, xl, yl))
            lp_bytes = st64["bytes_exec"] - (8 - vs) * (st64["points"] + a.n_cols + a.n_rows)
            res[f"spmv_{name}_ms"] = round(t, 4)
            res[f"spmv_{name}_speedup"] = round(t64 / t, 3)
            res[f"spmv_{name}_gbs"] = round(lp_bytes / (t * 1e-3) / 1e9, 1)
            res[f"spmv_{name}_relerr"] = relerr(yl.double().cpu().numpy(), ref_y)
            pl.destroy()
        del A
        q64 = ddf.ddf_inspect(*L, lo.n_cols, ddf.DDF_SPTRSV)
        tq = timed(lambda: ddf.ddf_sptrsv(q64, bd, xs))
        x64 = xs.cpu().numpy()
        res["sptrsv_f64_status"] = ddf.ddf_get_status(q64)
        q64.destroy()
        ref_x = refs[nm]["x"] if refs else x64
        res["sptrsv_f64_ms"] = round(tq, 4)
        res["sptrsv_f64_relerr"] = relerr(x64, ref_x)
        for dt, name in ((ddf.DDF_F32, "f32"), (ddf.DDF_BF16, "bf16")):
            ql = ddf.ddf_inspect(*L, lo.n_cols, ddf.DDF_SPTRSV, ddf.ddf_opts_default(store_dtype=dt))
            xr = torch.empty(lo.n_rows, dtype=torch.float64, device=dev)
            info = {}

            def go():
                info["r"] = ddf.ddf_sptrsv_refine(ql, bd, xr, tol=1e-12, max_iter=30)

            t = timed(go)
            st, iters, rel = info["r"]
            xh = xr.cpu().numpy()
            res[f"sptrsv_refine_{name}_ms"] = round(t, 4)
            res[f"sptrsv_refine_{name}_speedup"] = round(tq / t, 3)
            res[f"sptrsv_refine_{name}_iters"] = iters
            res[f"sptrsv_refine_{name}_relres_gpu"] = rel
            res[f"sptrsv_refine_{name}_status"] = st
            res[f"sptrsv_refine_{name}_relerr"] = relerr(xh, ref_x)
            if refs:
                res[f"sptrsv_refine_{name}_relres_oracle"] = oracle_relres(lo, xh, b)
            ql.destroy()
        del L
        out[nm] = res
    return out


def run_ablation(args, host, ddf, torch, dev, timed):
    """E5 (Sec. V, the BLAS-only comparison): plans restricted to BLAS codelets
    (plus PSC II, which covers whatever BLAS does not) against plans with every
    codelet type, executors timed alone.  Also E2's GPU recalibration of Eq. 1
    (ddf_tune_cost): the weight set it picks for each kernel, and the
    executors on plans mined with those weights."""
    out = {}
    td = lambda v: torch.from_numpy(np.ascontiguousarray(v)).to(dev)  # noqa: E731
    for nm in names(args.ablation):
        a, lo, x, b = host[nm] if nm in host else synth.workload(nm, args.scale)
        full = solo(ddf, torch, dev, timed, a, lo, x, b)
        ob = ddf.ddf_opts_default(allowed_types=ddf.DDF_ALLOW_BLAS | ddf.DDF_ALLOW_PSC2)
        bl = solo(ddf, torch, dev, timed, a, lo, x, b, ob, ob)
        oa, ka = ddf.ddf_tune_cost(td(a.rowptr), td(a.colidx), td(a.values), a.n_cols, ddf.DDF_SPMV)
        ol, kl = ddf.ddf_tune_cost(td(lo.rowptr), td(lo.colidx), td(lo.values), lo.n_cols, ddf.DDF_SPTRSV)
        tu = solo(ddf, torch, dev, timed, a, lo, x, b, oa, ol) if (ka or kl) else full
        out[nm] = {"all_types": {k: full[k] for k in ("spmv_ms", "spmv_gbs", "sptrsv_ms", "sptrsv_gbs",
                                                     "codelets_spmv", "ops_spmv", "codelets_sptrsv")},
                   "blas_psc2": {k: bl[k] for k in ("spmv_ms", "spmv_gbs", "sptrsv_ms", "sptrsv_gbs",
                                                   "codelets_spmv", "ops_spmv", "codelets_sptrsv")},
                   "spmv_speedup_all_vs_blas": round(bl["spmv_ms"] / full["spmv_ms"], 3),
                   "sptrsv_speedup_all_vs_blas": round(bl["sptrsv_ms"] / full["sptrsv_ms"], 3),
                   "eq1_tuned": {"spmv_weights": [oa.w_op, oa.w_codelet, oa.w_index],
                                 "sptrsv_weights": [ol.w_op, ol.w_codelet, ol.w_index],
                                 "spmv_ms": tu["spmv_ms"], "sptrsv_ms": tu["sptrsv_ms"],
                                 "spmv_speedup_vs_default": round(full["spmv_ms"] / tu["spmv_ms"], 3),
                                 "sptrsv_speedup_vs_default": round(full["sptrsv_ms"] / tu["sptrsv_ms"], 3)}}
    return out


def run_banded(args, ddf, torch, dev, timed, hbm, n=1 << 22, half_bw=8):
    """A band matrix of 17 nonzeros per row: its plan is BLAS codelets, so this
    times the BLAS SpMV kernel where it dominates."""
    m = synth.banded(max(1024, int(n * args.scale)), half_bw)
    x = synth.uniform_vector(m.n_cols, synth.SEED_BASE + 7)
    r = solo(ddf, torch, dev, timed, m, None, x, None, do_sptrsv=False)
    r["matrix"] = f"band, half bandwidth {half_bw}, N(0,1), diagonal 1 + sum |row|"
    r["spmv_frac_of_hbm"] = round(r["spmv_gbs"] / hbm, 4)
    return r


def run_e2e(args, D, ddf, torch, dev, stream, exec_b, world):
    """Same step from pinned host buffers: CSR, x and b copied in, y and x read back."""
    H = []
    h2d = d2h = 0
    for d in D:
        a, lo = d["a"], d["lo"]
        pin = lambda v: torch.from_numpy(np.ascontiguousarray(v)).pin_memory()  # noqa: E731
        H.append({"A": (pin(a.rowptr), pin(a.colidx), pin(a.values)),
                  "L": (pin(lo.rowptr), pin(lo.colidx), pin(lo.values)),
                  "x": pin(d["xh"]), "b": pin(d["bh"]),
                  "y": torch.empty(a.n_rows, dtype=torch.float64).pin_memory(),
                  "xs": torch.empty(lo.n_rows, dtype=torch.float64).pin_memory()})
        h2d += csr_bytes(a) + csr_bytes(lo) + 8 * a.n_cols + 8 * lo.n_rows
        d2h += 8 * a.n_rows + 8 * lo.n_rows

    # The chains (inspect(A) + spmv and inspect(L) + sptrsv of each matrix)
    # run on their own streams and host threads, as in the device-resident
    # step.  Uploads go on one copy stream, longest chain first (the L chains,
    # larger matrix first, then the A chains), and each chain's stream waits
    # only for its own arrays: the long solve chains start while the remaining
    # arrays are still being copied, instead of after all of them.
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


def oracle_spmv_cores(mats, reps=5):
    """The SpMV of the workload on the host: the sequential oracle (one core,
    the paper's baseline definition) and the row-parallel oracle over every
    host core; median of `reps`, GB/s of the executor's CSR bytes."""
    import oracle
    cores = os.cpu_count() or 1
    out = {"cores": cores}
    for key, fn in (("sequential", lambda a, x: oracle.spmv(a, x)),
                    ("parallel", lambda a, x: oracle.spmv_par(a, x, cores))):
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            for name, a, lo, x, b in mats:
                fn(a, x)
            ts.append(time.perf_counter() - t0)
        t = float(np.median(ts))
        byts = sum(12 * a.nnz + 4 * (a.n_rows + 1) + 8 * (a.n_cols + a.n_rows) for _, a, _, _, _ in mats)
        out[key] = {"ms": round(t * 1e3, 2), "gbs": round(byts / t / 1e9, 3)}
    return out


def oracle_references(args, host):
    """The CPU oracle's FP64 results for the mixed-precision matrices (part of
    the CPU-baseline leg): y = A x and the forward substitution of L x = b."""
    import oracle
    oracle.build()
    refs = {}
    for nm in names(args.mixed):
        a, lo, x, b = host[nm] if nm in host else synth.workload(nm, args.scale)
        refs[nm] = {"y": oracle.spmv_par(a, x), "x": oracle.sptrsv(lo, b)}
    return refs


def oracle_relres(lo, x, b):
    """||b - L x||_2 / ||b||_2 with the oracle's FP64 product."""
    import oracle
    r = b - oracle.spmv_par(lo, x)
    return float(np.linalg.norm(r) / np.linalg.norm(b))


def main(argv=None):
    args = parse(argv)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return 0
        mats = build_inputs(args.workload, args.scale)
        times = run_oracle(mats, 0, max_steps=args.steps, warmup=args.warmup)
        b = oracle_exec_bytes(mats)
        ms = 1e3 * float(np.mean(times))
        v = b / (ms * 1e-3) / 1e9
        line = {"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "GB/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(ms, 2), "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": args.workload, "scale": args.scale},
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
        mats = build_inputs(args.workload, args.scale)
        times = run_oracle(mats, args.cpu_seconds)
        b = oracle_exec_bytes(mats)
        cv = b / float(np.mean(times)) / 1e9
        cpu = {"value": round(cv, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
               "sample": f"{len(times)} full steps of the workload (sequential C oracle, "
                         f"{sum(times):.1f} s)", "exec_bytes_oracle_plan": b,
               "spmv_host_cores": oracle_spmv_cores(mats)}
    if rank == 0:
        hbm, _ = peaks()
        line = {
            "metric": METRIC, "value": round(r["value"], 2), "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(r["ms_per_step"], 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "scale": args.scale,
                       "step": "inspect(A)+spmv+inspect(L)+sptrsv per matrix",
                       "l2": "256 MB written then another 256 MB read between steps (the flush's "
                             "write-back happens before the timed work); inputs larger than L2",
                       "priorities": {"chain": "inspect(L)+sptrsv chains high, inspect(A)+spmv chains low",
                                      "achain": "inspect(A)+spmv chains high, inspect(L)+sptrsv chains low",
                                      "size": "both chains of the largest matrix high"}[args.prio],
                       "streams": {1: "everything on one stream",
                                   2: "one stream and host thread per matrix",
                                   4: "one stream and host thread per chain: inspect(A)+spmv, "
                                      "inspect(L)+sptrsv of each matrix"}[args.streams],
                       "parallelism": "replicas" if world > 1 else "single"},
            "frac_of_hbm": round(r["value"] / hbm, 4),
            "roofline": r["roofline"],
            "roofline_spmv": r["roofline_spmv"],
            "critical_path": r["critical_path"],
            "exec_only": r["exec_only"],
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
            "extra": r["extra"],
            "mixed_precision": r["mixed"],
            "ablation_e5": r["ablation"],
            "blas_banded": r["banded"],
            "batched": r["batched"],
            "exec_bytes_per_step": r["exec_bytes_per_step"],
        }
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
