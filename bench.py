"""Benchmark of the pair-counting hot path on GB300.

Workload (default): the light-cone xi(r, mu) configuration -- 500,000 data
objects in 20 clustered sky patches and 2,000,000 uniform randoms in the
shell r = 1000-2500, RA 0-60 deg, Dec 0-30 deg; 40 r bins on [0, 200) x 40 mu
bins on [0, 1] with the midpoint line of sight; DD, DR and RR, then the
Landy-Szalay estimator.  Synthetic, seeded (paper_1210_1833_gb300.synthetic).

One step = the whole hot path: catalog upload/conversion, cell-grid build
for both catalogs, the DD, DR and RR counts (one batched persistent launch
of the counting kernel), and the estimator.
`value` is pairs binned per second (pairs that fall in a bin of DD, DR or
RR) with the catalogs already in HBM; it does not depend on how many
candidate pairs the neighbour search examines.  The roofline is taken on the
counting launch, over the candidate pairs it evaluates.  `e2e` is the same step
through the public API from pinned host memory with the xi read back.  L2 is
flushed between timed steps.

--impl reference times the FP64 CPU oracle (the parity reference) on a
bounded sample of the same workload on the host cores.
"""
import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1210_1833_gb300 import synthetic  # noqa: E402

METRIC = "pairs/s & % FP32 roofline; batched/adjoint vs plain kernel, counts exact"
# Algorithmic FP32-pipe instructions per candidate pair, by separation
# measure: what the plain formula needs to separate, test and bin one pair
# (separation 3 FADD, squared norm FMUL + 2 FFMA, compare to the largest
# edge, scale and magic-number round to a bin index), plus the minimum image
# per axis (FADD + FMNMX) for periodic boxes, the second axis's index for
# (sigma, pi), and for (r, mu) the line of sight and the s.l, l.l products;
# theta on squared chords with a table index.  The kernel's own count (its
# near-edge tests and clamps included) is reported beside it from ncu.
I_PAIR = {"mono_open": 9, "mono_periodic": 15, "sigpi_periodic": 17, "rmu": 22, "theta": 10}
SM_COUNT = 152
FP32_LANES_PER_SM = 128


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.out = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index),
                                          "--query-gpu=" + q, "--format=csv,noheader,nounits",
                                          "-lms", "100"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def _cpu_model():
    """The host CPU's model name (for the CPU baseline's record)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip().lower() == "model name":
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def _kernel_hash():
    import glob
    import hashlib
    files = sorted(glob.glob(os.path.join(ROOT, "paper_1210_1833_gb300", "csrc", "count_*.cu*")) +
                   [os.path.join(ROOT, "paper_1210_1833_gb300", "csrc", f)
                    for f in ("cute_internal.h", "df_stage.h", "plan.cpp")])
    import re
    h = hashlib.sha256()
    for f in files:
        # the code only: comments and whitespace do not change the kernel
        src = open(f, encoding="utf-8").read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def _counters(key):
    """A kernel's ncu counters from profiles/counters.json, only if the
    counting-kernel sources still hash to what was captured."""
    path = os.path.join(ROOT, "profiles", "counters.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path)).get(key)
    if not rec or rec.get("kernel_source_hash") != _kernel_hash():
        return None
    return rec


def traffic_record(key):
    """DRAM bytes (read + write) per launch of a kernel, from ncu."""
    rec = _counters(key)
    return rec["per_launch_bytes"] if rec and "per_launch_bytes" in rec else None


def counted_record(key, cand_rate, peak):
    """The kernel's own FP32-pipe work per candidate pair, counted by ncu
    (scalar FADD/FMUL/FFMA thread instructions plus twice the packed ones,
    divided by the candidate pairs of the captured launch), and the FP32
    utilisation it implies at the measured rate; None once the kernel
    sources differ from the captured ones."""
    rec = _counters(key)
    if not rec or "fp32_ops_per_candidate" not in rec:
        return None
    i_c = rec["fp32_ops_per_candidate"]
    return {"i_pair": i_c, "frac": cand_rate * i_c / 1e12 / peak,
            "fma_pipe_active_pct": rec.get("fma_pipe_active_pct"),
            "source": "profiles/" + rec.get("summary", "")}


def total_pairs(nd, nr):
    return nd * (nd - 1) // 2 + nd * nr + nr * (nr - 1) // 2


# ------------------------------------------------------------------ reference arm
def cpu_oracle_rate(w, target_s=12.0, seed=0):
    """The oracle's cell-pruned FP64 mode (the exact-equivalent form of
    Sec. 3.3 that the CPU baseline times) on a bounded sample of the
    workload's pairs: a seeded subset of data rows against all randoms (DR).
    Returns (binned pairs/s, threads, sample description)."""
    import oracle
    nthr = oracle.max_threads()
    reach = [w.edges0[-1]] * 3
    rows = 256
    t = 0.0
    while True:
        sub = synthetic.subsample(w.data, rows, seed)
        t0 = time.perf_counter()
        c, _, _ = oracle.count(w.kind, sub, w.randoms, edges0=w.edges0, edges1=w.edges1,
                               periodic=w.periodic, L=w.L, cells=reach)
        t = time.perf_counter() - t0
        if t >= target_s / 3 or rows >= len(w.data):
            break
        rows = int(min(len(w.data), rows * max(2.0, min(8.0, target_s / max(t, 1e-3)))))
    binned = int(c.sum())
    return binned / t, nthr, ("%d data rows x %d randoms (DR, cell-pruned FP64 oracle on "
                              "cells of the reach: %d binned pairs in %.1f s, grid build "
                              "included)" % (rows, len(w.randoms), binned, t))


def run_reference(args, w, rank, world):
    if rank != 0:
        return
    import oracle  # noqa: F401
    vals, times = [], []
    desc = ""
    thr = 0
    for _ in range(args.warmup):
        cpu_oracle_rate(w, target_s=3.0)
    for _ in range(args.steps):
        t0 = time.perf_counter()
        v, thr, desc = cpu_oracle_rate(w, target_s=8.0)
        times.append((time.perf_counter() - t0) * 1e3)
        vals.append(v)
    v = float(np.median(vals))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "pairs/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": float(np.median(times)), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(workload_config(w), sample="each step a bounded DR sample (below)"),
            "cpu_baseline": {"value": v, "unit": "pairs/s", "cores": thr, "kind": "oracle",
                             "cpu": _cpu_model(), "sample": desc},
            "e2e": {"value": v, "unit": "pairs/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_config(w):
    """The workload part of the JSON config, shared by both arms."""
    return {"workload": w.name, "kind": w.kind, "n_data": len(w.data), "n_randoms": len(w.randoms),
            "bins": [len(w.edges0) - 1, len(w.edges1) - 1], "counts": ["DD", "DR", "RR"],
            "estimator": "landy-szalay"}


# ------------------------------------------------------------------ GPU arm
def run_gpu(args, w, rank, world):
    import torch
    from paper_1210_1833_gb300 import cute
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    ctx = cute.Context(dev)
    ctx.set_timing(True)
    nd, nr = len(w.data), len(w.randoms)
    reach = [w.edges0[-1]] * 3
    d_dev = torch.from_numpy(w.data).to(f"cuda:{dev}")
    r_dev = torch.from_numpy(w.randoms).to(f"cuda:{dev}")
    d_pin = torch.from_numpy(w.data).pin_memory()
    r_pin = torch.from_numpy(w.randoms).pin_memory()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=f"cuda:{dev}")  # 256 MB
    # (rr_*: the counting launch the roofline is taken on, all of the step's
    # counts in one launch)
    state = {"cand": 0, "kms": [], "rr_cand": 0, "rr_ms": [], "inrange": 0, "rechecked": 0, "fp64": 0,
             "slots": 0, "per": {}, "stencil": 0}

    names = [n for n in ("DD", "DR", "RR") if not args.only or n in args.only.split(",")]
    label = "+".join(names)

    def step(dsrc, rsrc, record):
        cd = ctx.upload(dsrc)
        cr = ctx.upload(rsrc)
        ctx.grid([cd, cr], reach, args.cpr)
        sets = {"DD": (cd, None), "DR": (cd, cr), "RR": (cr, None)}
        # the step's counts in one persistent launch (one work list, one
        # round trip, one tail): the library's batched call
        got = ctx.count_batched("rmu", [sets[n] for n in names], w.edges0, w.edges1)
        res = {n: np.ones((len(w.edges0) - 1, len(w.edges1) - 1), np.uint64)
               for n in ("DD", "DR", "RR")}
        res.update(dict(zip(names, got)))
        if record:
            st = ctx.stats()
            state["cand"] += st["candidate_pairs"]
            state["stencil"] += st["stencil_pairs"]
            state["kms"].append(st["kernel_ms"])
            state["per"].setdefault(label, []).append(st["kernel_ms"])
            state["rechecked"] += st["rechecked_pairs"]
            state["fp64"] += st["fp64_pairs"]
            state["slots"] += st["pair_slots"]
            state["inrange"] += int(sum(int(c.sum()) for c in got))
            state["rr_cand"] = st["candidate_pairs"]
            state["rr_ms"].append(st["kernel_ms"])
        xi = cute.estimator("ls", res["DD"], res["DR"], res["RR"], nd, nr)
        cd.free()
        cr.free()
        return xi

    def timed(dsrc, rsrc, steps, record):
        times = []
        for _ in range(steps):
            flush.zero_()
            torch.cuda.synchronize()
            if world > 1:
                torch.distributed.barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(dsrc, rsrc, record)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        return times

    for _ in range(args.warmup):
        step(d_dev, r_dev, False)
    torch.cuda.synchronize()
    tuning = {}
    if args.tune:
        # cells per reach by whole steps, then each count's launch shape by
        # the library's autotuner (remembered per problem shape, so the
        # re-uploaded catalogs of the timed steps use it)
        best = None
        for cpr in (3, 4, 5):
            args.cpr = cpr
            step(d_dev, r_dev, False)
            dts = []
            for _ in range(2):  # the faster of two: one step is noisy at the 1 % level
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                step(d_dev, r_dev, False)
                torch.cuda.synchronize()
                dts.append(time.perf_counter() - t0)
            if best is None or min(dts) < best[0]:
                best = (min(dts), cpr)
        args.cpr = best[1]
        # then the launch's home objects per lane and neighbour slice, also
        # by whole steps (a sample of work items misjudges the neighbour
        # cull, which culls less around wider home chunks)
        best = None
        for hp in (2, 4):
            for sl in (1024, 4096):
                ctx.set_launch(home_per_lane=hp, slice=sl)
                dts = []
                for _ in range(2):
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    step(d_dev, r_dev, False)
                    torch.cuda.synchronize()
                    dts.append(time.perf_counter() - t0)
                if best is None or min(dts) < best[0]:
                    best = (min(dts), hp, sl)
        ctx.set_launch(home_per_lane=best[1], slice=best[2])
        tuning[label] = {"home_per_lane": best[1], "slice": best[2],
                         "warps_per_block": "library default", "by": "whole steps"}
        tuning["cells_per_reach"] = args.cpr
        step(d_dev, r_dev, False)
        torch.cuda.synchronize()
    clk = ClockSampler(dev)
    clk.start()
    t_dev = timed(d_dev, r_dev, args.steps, True)
    # one untimed step through the host buffers first: the first GPU access
    # to newly pinned memory costs once, not per step (the device-resident
    # steps had their warm-up above)
    step(d_pin, r_pin, False)
    torch.cuda.synchronize()
    t_e2e = timed(d_pin, r_pin, max(1, args.steps // 2), False)
    clocks = clk.stop()
    ms = float(np.sum(t_dev)) / len(t_dev)
    ms_e2e = float(np.sum(t_e2e)) / len(t_e2e)
    if world > 1:
        t = torch.tensor([ms, ms_e2e], device=f"cuda:{dev}")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms, ms_e2e = float(t[0]), float(t[1])
    cand_per_step = state["cand"] / args.steps
    inrange_per_step = state["inrange"] / args.steps
    value = world * inrange_per_step / (ms / 1e3)
    e2e_value = world * inrange_per_step / (ms_e2e / 1e3)
    if rank != 0:
        return
    pk, src = peaks()
    smax = float(pk.get("sm_max_mhz", 2070.0))
    peak_tinst = SM_COUNT * FP32_LANES_PER_SM * smax * 1e6 / 1e12
    rr_ms = float(np.mean(state["rr_ms"])) if state["rr_ms"] else float("nan")
    rr_rate = state["rr_cand"] / (rr_ms / 1e3)
    achieved = rr_rate * I_PAIR["rmu"] / 1e12
    if args.no_cpu:
        cpu_v, cpu_thr, cpu_desc = None, None, "skipped (--no-cpu)"
    else:
        cpu_v, cpu_thr, cpu_desc = cpu_oracle_rate(w, target_s=12.0)
    # upload stats x2; grid x2 (assign, 3 scan passes, scatter); the work
    # list (entry counts, 2 scan passes, record write) and the one counting
    # launch of DD, DR and RR
    launches_per_step = 2 + 2 * 5 + 5
    line = {
        "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {**workload_config(w), "l2": "flushed between steps (256 MB write)",
                   "parallelism": "replicas" if world > 1 else "single",
                   "cells_per_reach": args.cpr, "autotuned": tuning or None},
        "pairs": {"candidate_per_step": cand_per_step,
                  "stencil_per_step": state["stencil"] / args.steps,
                  "in_range_per_step": inrange_per_step,
                  "all_pairs_per_step": total_pairs(nd, nr),
                  "candidate_pairs_per_s": world * cand_per_step / (ms / 1e3),
                  "stencil_pairs_per_s": world * state["stencil"] / args.steps / (ms / 1e3),
                  "all_pairs_per_s": world * total_pairs(nd, nr) / (ms / 1e3),
                  "count_kernel_ms": {k: float(np.mean(v)) for k, v in state["per"].items()},
                  "rechecked_fraction": state["rechecked"] / max(1, state["cand"]),
                  "fp64_fraction": state["fp64"] / max(1, state["cand"]),
                  "slot_utilisation": state["cand"] / max(1, state["slots"]),
                  "count_kernel_ms_per_step": float(np.sum(state["kms"])) / args.steps},
        "roofline": {"bound": "alu", "kernel": "k_count<R_MU> (%s, one launch)" % label,
                     "achieved": achieved,
                     "peak": peak_tinst, "unit": "Tinst/s", "frac": achieved / peak_tinst,
                     "traffic": traffic_record("k_count_rmu_c2_step" if label == "DD+DR+RR"
                                               else "k_count_rmu_RR_c2"),
                     "i_pair": I_PAIR["rmu"],
                     "counted": counted_record("k_count_rmu_RR_c2", rr_rate, peak_tinst),
                     "peak_note": "152 SMs x 128 FP32 lanes x %.0f MHz (%s max clock)" % (
                         smax, src),
                     "kernel_ms": rr_ms, "candidate_pairs": state["rr_cand"]},
        "cpu_baseline": {"value": cpu_v, "unit": "pairs/s", "cores": cpu_thr, "kind": "oracle",
                         "cpu": _cpu_model(), "sample": cpu_desc},
        "e2e": {"value": e2e_value, "unit": "pairs/s", "ms_per_step": ms_e2e,
                "h2d_bytes_per_step": int(w.data.nbytes + w.randoms.nbytes),
                "d2h_bytes_per_step": int(3 * 8 * (len(w.edges0) - 1) * (len(w.edges1) - 1))},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
    }
    if not args.no_extras and not args.only:
        ctx.set_launch()  # the rows take their own launch shapes
        line["rows"] = run_extras(ctx, dev)
    print(json.dumps(line), flush=True)
    ctx.close()


def run_extras(ctx, dev, reps=3, which="all"):
    """The other rows of the path, measured beside the plain kernel:
    batched xi(sigma, pi) of 64 periodic boxes in one persistent launch
    (replayed CUDA graph) vs 192 separate counts, and the weighted forward
    and the adjoint of 4M weighted objects vs the plain count."""
    import torch
    stream = torch.cuda.current_stream(dev)

    def timed(fn, n=reps):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    out = {}
    rows = [("batched", _row_batched), ("weighted", _row_weighted), ("monopole", _row_monopole),
            ("density", _row_density), ("pixel", _row_pixel), ("angular", _row_angular)]
    for name, fn in rows:
        if which not in ("all", name):
            continue
        try:
            out.update(fn(ctx, dev, timed))
        except Exception as e:  # a failed row is reported, the headline line still prints
            out[name] = {"error": "%s: %s" % (type(e).__name__, e)}
    return out


_ROW_TUNE = True  # --no-tune: the rows' counts keep the library's default launch shape
_ROW_SCALE = 1.0  # --row with --scale: a smaller copy of the row's workload (profiling)


def _row_batched(ctx, dev, timed):
    import torch
    out = {}
    # (--row batched --scale s: the first 64 s boxes, for profiling)
    boxes = synthetic.c4_batched_sigpi(n_boxes=max(1, int(round(64 * _ROW_SCALE))))
    e0, e1 = boxes[0].edges0, boxes[0].edges1
    reach = [e0[-1], e0[-1], e1[-1]]
    cats, pairs = [], []
    for b in boxes:
        d = ctx.upload(b.data, periodic=True, L=b.L)
        r = ctx.upload(b.randoms, periodic=True, L=b.L)
        ctx.grid([d, r], reach)  # cells per reach from the density
        cats.append((d, r))
        pairs += [(d, None), (d, r), (r, None)]
    nb = (len(e0) - 1) * (len(e1) - 1)
    plain_out = [torch.zeros(nb, dtype=torch.int64, device=f"cuda:{dev}") for _ in pairs]

    def batched():
        ctx.count_batched("sigpi", pairs, e0, e1, device=True)

    def plain():
        for (a, b), o in zip(pairs, plain_out):
            ctx.count("sigpi", a, b, e0, e1, out=o, want_oor=False)

    # both paths once before either is timed (work lists, graph capture,
    # clocks up from idle)
    batched()
    plain()
    t_b = timed(batched)
    t_p = timed(plain)
    batched()
    torch.cuda.synchronize()
    st = ctx.stats()
    binned = sum(int(c.sum()) for c in ctx.count_batched("sigpi", pairs, e0, e1, device=True))
    name = "batched_sigpi_64_boxes" if len(boxes) == 64 else "batched_sigpi_%d_boxes" % len(boxes)
    out[name] = {
        "batched_ms": t_b, "plain_ms": t_p, "plain_over_batched": t_p / t_b,
        "launches": {"batched": 1, "plain": len(pairs)}, "binned_pairs": binned,
        "binned_pairs_per_s": binned / (t_b / 1e3), "graph_replay": True,
        "batched_candidate_pairs": st["candidate_pairs"], "batched_kernel_ms": st["kernel_ms"],
        "batched_recheck": _recheck(st),
        "batched_roofline": _alu_roofline(st["candidate_pairs"] / (st["kernel_ms"] / 1e3),
                                          "sigpi_periodic")}
    for d, r in cats:
        d.free(); r.free()
    return out


def _recheck(st):
    """Fractions of a count's candidate pairs that were re-tested near an
    edge, and that the FP64 formula decided (re-tested pairs the
    double-float stage could not settle)."""
    c = max(1, int(st.get("candidate_pairs", 0)))
    return {"rechecked_fraction": int(st.get("rechecked_pairs", 0)) / c,
            "fp64_fraction": int(st.get("fp64_pairs", 0)) / c}


def _alu_roofline(cand_rate, kind):
    """Algorithmic FP32 roofline fraction of a counting kernel."""
    pk, src = peaks()
    peak = SM_COUNT * FP32_LANES_PER_SM * float(pk.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
    ach = cand_rate * I_PAIR[kind] / 1e12
    return {"bound": "alu", "i_pair": I_PAIR[kind], "achieved": ach, "peak": peak,
            "unit": "Tinst/s", "frac": ach / peak}


def _row_monopole(ctx, dev, timed):
    """c1: monopole DD of 20,000 points in a periodic box, against its
    algorithmic roofline: step_ms is grid build + count per call, count_ms
    the count alone on the built grid."""
    import torch
    w = synthetic.c1_monopole_box()
    A = ctx.upload(w.data, periodic=True, L=w.L)
    cnt = torch.zeros(len(w.edges0) - 1, dtype=torch.int64, device=f"cuda:{dev}")

    cpr = [0]  # cells per reach: the library's density choice unless tuned

    def step():
        ctx.grid([A], [w.edges0[-1]] * 3, cpr[0])
        ctx.count("mono", A, None, w.edges0, out=cnt, want_oor=False)

    # a small count: let the autotuner pick the cell size, home objects,
    # warps and slice
    ctx.grid([A], [w.edges0[-1]] * 3)
    tuned = (ctx.autotune("mono", [(A, None)], w.edges0, tune_cells=True, max_items=1 << 30)
             if _ROW_TUNE else None)
    if tuned:
        cpr[0] = tuned["cells_per_reach"]
    t = timed(step)
    st = ctx.stats()

    # the count alone on the built grid (its work list cached): what a call
    # costs beside the kernel when the grid is reused
    def count_only():
        ctx.count("mono", A, None, w.edges0, out=cnt, want_oor=False)

    t_count = timed(count_only, 20)
    out = {"monopole_c1_20k": {
        "step_ms": t, "count_ms": t_count, "count_over_kernel": t_count / st["kernel_ms"],
        "kernel_ms": st["kernel_ms"], "candidate_pairs": st["candidate_pairs"],
        "binned_pairs": int(cnt.sum()), "tuned": tuned, "recheck": _recheck(st),
        "roofline": _alu_roofline(st["candidate_pairs"] / (st["kernel_ms"] / 1e3),
                                  "mono_periodic")}}
    A.free()
    return out


def _row_density(ctx, dev, timed):
    """Density-grid monopole of the c5 box (4M weighted objects, L = 2000):
    TSC to 256^3, lag correlations to r = 150 (30 bins); one FP32 FMA per
    (grid point, lag) pair is the algorithmic work."""
    import torch
    w = synthetic.c5_weighted()
    x = torch.from_numpy(w.data).to(f"cuda:{dev}")
    wt = torch.from_numpy(w.weights).to(f"cuda:{dev}")
    ng = 256
    res = {}
    t = timed(lambda: res.__setitem__("v", ctx.density_grid_xi(x, w.L, ng, w.edges0, weights=wt)))
    kms = ctx.stats()["kernel_ms"]  # the lag-correlation kernel alone
    lags = float(res["v"][1].sum())
    fma = lags * ng ** 3
    pk, src = peaks()
    peak = SM_COUNT * FP32_LANES_PER_SM * float(pk.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
    return {"density_grid_c5_256": {
        "call_ms": t, "lag_kernel_ms": kms, "grid": ng, "lags": lags, "fma": fma,
        "roofline": {"bound": "alu", "i_per_unit": 1, "unit_of_work": "grid point x lag",
                     "achieved": fma / (kms / 1e3) / 1e12, "peak": peak, "unit": "Tinst/s",
                     "frac": fma / (kms / 1e3) / 1e12 / peak,
                     "note": "lag-correlation kernel (CUDA events); the call adds TSC, "
                             "overdensity and binning"}}}


def _row_pixel(ctx, dev, timed):
    """w_pix: the c3 data (5M unit vectors) as a HEALPix nside 1024 map,
    its occupied pixels correlated with their counts as weights."""
    import torch
    from paper_1210_1833_gb300 import cute
    w = synthetic.c3_angular()
    chord = cute.theta_to_chord(w.extra["theta_deg"])
    x = torch.from_numpy(w.data).to(f"cuda:{dev}")
    ns = 1024
    state = {}

    def make_map():
        m = ctx.pixel_map(x, None, ns)
        pix = torch.nonzero(m).view(-1)
        state["cen"] = ctx.pixel_centres(ns, pix)
        state["wt"] = m[pix].to(torch.float32)

    t_map = timed(make_map)
    P = ctx.upload(state["cen"], weights=state["wt"])
    ctx.grid([P], [chord[-1]] * 3)
    cnt = torch.zeros(len(chord) - 1, dtype=torch.int64, device=f"cuda:{dev}")
    ws = torch.zeros(len(chord) - 1, dtype=torch.float64, device=f"cuda:{dev}")
    t_cnt = timed(lambda: ctx.count("theta", P, None, chord, weighted=True, out=cnt,
                                    wsum_out=ws, want_oor=False))
    st = ctx.stats()
    out = {"pixel_map_c3_nside1024": {
        "objects": len(w.data), "pixels": int(state["cen"].shape[0]), "map_ms": t_map,
        "weighted_count_ms": t_cnt, "kernel_ms": st["kernel_ms"],
        "candidate_pairs": st["candidate_pairs"], "recheck": _recheck(st),
        "roofline": _alu_roofline(st["candidate_pairs"] / (st["kernel_ms"] / 1e3), "theta")}}
    P.free()
    return out


def _row_angular(ctx, dev, timed):
    """c3: w(theta) DD, DR and RR of 5M data and 20M randoms on a 1000 sq-deg
    cap (64 log theta bins, binned on chords), each count timed once (CUDA
    events around the kernel) after a warm-up count on a 2% sample; the
    largest workload, whose step (about a minute) is too long to repeat as
    the headline's timed steps."""
    w = synthetic.c3_angular(scale=_ROW_SCALE)
    from paper_1210_1833_gb300 import cute
    chord = cute.theta_to_chord(w.extra["theta_deg"])
    D, R = ctx.upload(w.data), ctx.upload(w.randoms)
    S = ctx.upload(w.data[: len(w.data) // 50])
    ctx.grid([D, R, S], [chord[-1]] * 3)
    ctx.count("theta", S, None, chord, want_oor=False)
    res = {}
    for name, a, b in (("DD", D, None), ("DR", D, R), ("RR", R, None)):
        c, _, _ = ctx.count("theta", a, b, chord, want_oor=False)
        st = ctx.stats()
        res[name] = {"kernel_ms": st["kernel_ms"], "candidate_pairs": st["candidate_pairs"],
                     "stencil_pairs": st["stencil_pairs"],
                     "binned_pairs": int(c.sum()), "recheck": _recheck(st),
                     "roofline": _alu_roofline(st["candidate_pairs"] / (st["kernel_ms"] / 1e3),
                                               "theta")}
    for c in (D, R, S):
        c.free()
    tot_ms = sum(v["kernel_ms"] for v in res.values())
    binned = sum(v["binned_pairs"] for v in res.values())
    res["step"] = {"count_kernel_ms": tot_ms, "binned_pairs": binned,
                   "binned_pairs_per_s": binned / (tot_ms / 1e3),
                   "candidate_pairs_per_s": sum(v["candidate_pairs"] for v in res.values()) /
                   (tot_ms / 1e3), "n_data": len(w.data), "n_randoms": len(w.randoms)}
    name = "angular_c3_5M_20M" if _ROW_SCALE == 1.0 else "angular_c3_scale%g" % _ROW_SCALE
    return {name: res}


def _row_weighted(ctx, dev, timed):
    import torch
    out = {}
    w = synthetic.c5_weighted()
    e = w.edges0
    A = ctx.upload(w.data, weights=w.weights, periodic=True, L=w.L)
    ctx.grid([A], [e[-1]] * 3)  # cells per reach from the density
    cnt = torch.zeros(len(e) - 1, dtype=torch.int64, device=f"cuda:{dev}")
    ws = torch.zeros(len(e) - 1, dtype=torch.float64, device=f"cuda:{dev}")
    G = torch.from_numpy(w.extra["G"]).to(f"cuda:{dev}")
    tuned = (ctx.autotune("mono", [(A, None)], e, tune_cells=False, max_items=30000)
             if _ROW_TUNE else None)
    t_plain = timed(lambda: ctx.count("mono", A, None, e, out=cnt, want_oor=False))
    st = ctx.stats()
    t_w = timed(lambda: ctx.count("mono", A, None, e, weighted=True, out=cnt, wsum_out=ws,
                                  want_oor=False))
    t_adj = timed(lambda: ctx.adjoint("mono", A, None, e, G=G))
    binned = int(cnt.sum())
    out["weighted_adjoint_4M"] = {
        "plain_ms": t_plain, "weighted_ms": t_w, "adjoint_ms": t_adj,
        "weighted_over_plain": t_w / t_plain, "adjoint_over_plain": t_adj / t_plain,
        "binned_pairs": binned, "plain_binned_pairs_per_s": binned / (t_plain / 1e3),
        "plain_candidate_pairs": st["candidate_pairs"], "plain_kernel_ms": st["kernel_ms"],
        "plain_home_per_lane": st["home_per_lane"], "plain_tuned": tuned,
        "plain_recheck": _recheck(st),
        "plain_candidate_pairs_per_s": st["candidate_pairs"] / (st["kernel_ms"] / 1e3),
        "plain_roofline": _alu_roofline(st["candidate_pairs"] / (st["kernel_ms"] / 1e3),
                                        "mono_periodic")}
    A.free()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--scale", type=float, default=1.0, help="workload scale (1 = full size)")
    ap.add_argument("--only", default="", help="profiling: run only these counts (e.g. RR)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the timed CPU oracle sample")
    ap.add_argument("--cpr", type=int, default=4, help="cells per reach of the grid")
    ap.add_argument("--no-tune", dest="tune", action="store_false",
                    help="skip the warm-up autotuning (cells per reach, launch shapes)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched / weighted / adjoint measurements")
    ap.add_argument("--row", default="",
                    choices=["", "batched", "weighted", "monopole", "density", "pixel", "angular"],
                    help="profiling: run only this row and print it (with --scale, the "
                         "angular row on a smaller copy of its workload)")
    args = ap.parse_args()
    global _ROW_TUNE, _ROW_SCALE
    _ROW_TUNE = args.tune
    if args.row:
        _ROW_SCALE = args.scale
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl == "gb300" else "gloo")
    if args.row and args.impl == "gb300":
        import torch
        from paper_1210_1833_gb300 import cute
        dev = int(os.environ.get("LOCAL_RANK", "0"))
        torch.cuda.set_device(dev)
        ctx = cute.Context(dev)
        ctx.set_timing(True)
        print(json.dumps(run_extras(ctx, dev, reps=max(1, args.steps), which=args.row)), flush=True)
        ctx.close()
        return
    w = synthetic.c2_rmu_lightcone(scale=args.scale)
    if args.impl == "reference":
        run_reference(args, w, rank, world)
    else:
        run_gpu(args, w, rank, world)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
