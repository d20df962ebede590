#!/usr/bin/env python
"""Benchmark of s-line graph construction on one GB300 (or N replicas).

Workload: the medium synthetic hypergraph (m = 1,000,000 hyperedges over
n = 500,000 vertices, log-normal(1.8, 1.0) sizes clipped to [2, 5000],
Zipf(1.7) vertex popularity, seed 0) with the sweep s = 1..8.

One step = the whole hot path on that input, resident in HBM:
  slg_load from device memory (validate, transpose), then the sweep as one
  ensemble (Algorithm 3: one plan and one counting pass for every s), then for
  every s its window plan and the fill of every window of at most 2^33 pairs
  into a reused device window. `--sweep per_s` runs each s on its own instead
  (plan, counting pass, windows).
Metric: wedges per second, W = sum_s W_s with W_s = sum_v C(d_s(v), 2);
s-edges per second (sum_s |L_s| / time) is reported beside it.

Prints one JSON line (rank 0). `--impl reference` times the CPU oracle on a
bounded row sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

WORKLOAD = ("medium: m=1,000,000 hyperedges, n=500,000 vertices, sizes log-normal(1.8,1.0) "
            "clipped [2,5000], vertex popularity Zipf(1.7), seed 0; s=1..8 sweep")
METRIC = "s-line wedges/s (medium hypergraph, s=1..8, bit-exact)"
WINDOW = 1 << 33          # default pairs per output window (96 GiB of I/J/O)
L2_FLUSH_BYTES = 512 << 20


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--s", default="1-8", help="s values, e.g. 1-8 or 2,4")
    ap.add_argument("--m", type=int, default=1_000_000, help="hyperedges (default: full size)")
    ap.add_argument("--cpu-rows", type=int, default=600, help="rows in the CPU-oracle sample")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--window", type=int, default=WINDOW, help="pairs per output window")
    ap.add_argument("--workload", choices=["medium", "large", "batch", "serve", "ensemble"],
                    default="medium")
    ap.add_argument("--graphs", type=int, default=4096, help="batch workload: number of graphs")
    ap.add_argument("--sweep", choices=["ensemble", "stream", "per_s"], default=None,
                    help="the s sweep as one ensemble (medium default), as one-walk windows of "
                         "every list (large default), or one s at a time")
    ap.add_argument("--ens-windows", choices=["per_list", "all"], default=None,
                    help="--sweep ensemble: each list in its own windows (the medium "
                         "default), or windows of every list, the later lists filtered from the "
                         "one before where that reads less (the large default)")
    ap.add_argument("--queries", type=int, default=1000, help="serve workload: queries per rate")
    ap.add_argument("--degree-cap", type=int, default=100_000,
                    help="large workload: cap on the Chung-Lu target degree (scale it with --m "
                         "to keep the density of the hub lists, e.g. 6000 at m=2,000,000)")
    return ap.parse_args()


def s_values(spec: str):
    out = []
    for part in spec.split(","):
        if "-" in part:
            a, b = part.split("-")
            out.extend(range(int(a), int(b) + 1))
        else:
            out.append(int(part))
    return out


def workload(m: int):
    key = f"medium_m{m}_seed0"
    return synth.cached(key, lambda: synth.medium(seed=0, m=m))


LARGE_WORKLOAD = ("large hub-heavy: m=20,000,000 hyperedges, n=10,000,000 vertices, sizes "
                  "log-normal(2.0,1.1) clipped [2,20000], Chung-Lu popularity with vertex degree "
                  "Zipf(1.8) capped at 100,000, seed 0; s in {2,4,8,16}")
LARGE_METRIC = "s-line wedges/s (large hub-heavy hypergraph, s in {2,4,8,16}, bit-exact)"


def workload_spec(args):
    """(graph, s list, workload text, metric, CPU-oracle rows) of the timed workload."""
    if args.workload == "large":
        m = args.m if args.m != 1_000_000 else 20_000_000
        cap = getattr(args, "degree_cap", 100_000)
        if cap == 100_000:
            h = synth.cached(f"large_m{m}_seed0", lambda: synth.large(seed=0, m=m))
        else:
            h = synth.cached(f"large_m{m}_cap{cap}_seed0", lambda: synth.build(
                (0,), m, m // 2, "lognormal", (2.0, 1.1, 2, 20000), "chung_lu", (1.8, cap),
                f"large_m{m}_cap{cap}", fast=True))
        s_list = [2, 4, 8, 16] if args.s == "1-8" else s_values(args.s)
        text = LARGE_WORKLOAD if m == 20_000_000 else f"{LARGE_WORKLOAD} (m={m})"
        if cap != 100_000:
            text += f" (degree cap {cap})"
        # rows of the large graph meet 20x more partners: a 40-row sample keeps the
        # CPU baseline to seconds
        return h, s_list, text, LARGE_METRIC, (40 if args.cpu_rows == 600 else args.cpu_rows)
    h = workload(args.m)
    text = WORKLOAD if args.m == 1_000_000 else f"{WORKLOAD} (m={args.m})"
    return h, s_values(args.s), text, METRIC, args.cpu_rows


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# --------------------------------------------------------------- CPU oracle

def oracle_sample(h, s_list, rows: int, seed: int):
    """Time the CPU oracle on `rows` random rows (all s at once)."""
    import oracle
    rng = np.random.default_rng([seed, 5])
    sample = np.sort(rng.choice(h.m, size=min(rows, h.m), replace=False)).astype(np.int32)
    cores = host_cores()
    t0 = time.perf_counter()
    _, _, osum = oracle.rows(h.off, h.idx, sample, s_list, nthreads=cores)
    dt = time.perf_counter() - t0
    wedges = int(osum.sum())
    return wedges, dt, cores, f"{sample.size} random rows (seed {seed}) x s={s_list[0]}..{s_list[-1]}"


# ------------------------------------------------------------------- clocks

class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.path = os.path.join(tempfile.gettempdir(), f"slg_clocks_{os.getpid()}.csv")
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        # samples under load: the upper half by clock (idle gaps between kernels read low)
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------- GPU step

def run_sweep(slg, g, s_list, bufs, stream, per_s, mode_work=None):
    """Counting pass + windowed fill for every s on a loaded graph. With
    mode_work, each s's per-handler work is recorded after its counting pass."""
    import torch
    I, J, O = bufs
    WINDOW = I.numel()
    for s in s_list:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pairs, wedges = slg.slg_count(g, s)
        if mode_work is not None:
            mode_work[s] = slg.slg_mode_stats(g, s)
        splits = slg.slg_plan_windows(g, s, WINDOW)
        for r0, r1 in zip(splits[:-1], splits[1:]):
            slg.slg_build_window(g, s, int(r0), int(r1), I, J, O, WINDOW)
        e1.record(stream)
        e1.synchronize()
        d = per_s.setdefault(s, {"s": s, "wedges": wedges, "pairs": pairs, "ms": []})
        d["ms"].append(e0.elapsed_time(e1))


def run_sweep_ensemble(slg, g, s_list, bufs, stream, per_s, wedges, mode_work=None,
                       all_lists=False, made=None):
    """The s sweep as one ensemble (Algorithm 3): one plan for min(s) and one
    counting pass for every list, then each list's windows (per s: its fill time),
    or windows holding every list (all_lists: the later lists filtered from the
    one before where that reads less; per s: its filters' time, measured, plus
    its share of the walking fills, in proportion to the pairs they wrote). The
    shared counting pass is charged to the lists in equal parts. made (per s:
    windows walked, pairs walked, windows filtered, pairs filtered, filter
    microseconds, pairs the filter read) accumulates slg_ensemble_fill_stats."""
    import torch
    I, J, O = bufs
    cap = I.numel()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(s_list) + 2)]
    ev[0].record(stream)
    pairs, _ = slg.slg_ensemble_count(g, s_list)
    ev[1].record(stream)
    if mode_work is not None:
        for t, s in enumerate(s_list):
            mode_work[s] = slg.slg_ensemble_mode_stats(g, s_list, t)
    if all_lists:
        splits = slg.slg_ensemble_plan_windows(g, s_list, cap, which=slg.ENSEMBLE_ALL)
        for r0, r1 in zip(splits[:-1], splits[1:]):
            slg.slg_ensemble_build_window(g, s_list, int(r0), int(r1), I, J, O, cap,
                                          which=slg.ENSEMBLE_ALL)
        ev[-1].record(stream)
    else:
        for t, s in enumerate(s_list):
            splits = slg.slg_ensemble_plan_windows(g, s_list, cap, which=t)
            for r0, r1 in zip(splits[:-1], splits[1:]):
                slg.slg_ensemble_build_window(g, s_list, int(r0), int(r1), I, J, O, cap, which=t)
            ev[t + 2].record(stream)
    ev[-1].synchronize()
    count_ms = ev[0].elapsed_time(ev[1])
    fill_all = ev[1].elapsed_time(ev[-1])
    fs = slg.slg_ensemble_fill_stats(g, reset=True)
    if made is not None:
        for t, s in enumerate(s_list):
            acc = made.setdefault(s, [0] * 6)
            for c in range(6):
                acc[c] += int(fs[t][c])
    filt_ms = [fs[t][4] / 1e3 for t in range(len(s_list))]
    walked = max(sum(int(fs[t][1]) for t in range(len(s_list))), 1)
    walk_ms = max(fill_all - sum(filt_ms), 0.0)
    for t, s in enumerate(s_list):
        d = per_s.setdefault(s, {"s": s, "wedges": wedges[s], "pairs": pairs[t], "ms": [],
                                 "fill_ms": [], "count_ms_shared": [], "filter_ms": []})
        fill = (filt_ms[t] + walk_ms * int(fs[t][1]) / walked if all_lists
                else ev[t + 1].elapsed_time(ev[t + 2]))
        d["filter_ms"].append(filt_ms[t])
        d["fill_ms"].append(fill)
        d["count_ms_shared"].append(count_ms)
        d["ms"].append(fill + count_ms / len(s_list))


def run_sweep_stream(slg, g, s_list, bufs, stream, per_s, wedges, mode_work=None, made=None):
    """The s sweep as one-walk windows of every list (slg_ensemble_stream_window):
    no counting pass over the whole graph; each window's sparse-accumulator and
    hub-pair rows are walked once, the later lists filtered from the one before.
    Per s: its filters' time (measured) for s after the first; the rest of the
    step for the first. made accumulates slg_ensemble_fill_stats."""
    import torch
    I, J, O = bufs
    cap = I.numel()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    tot = [0] * len(s_list)
    r0 = 0
    while r0 < g.m:
        r0, pairs = slg.slg_ensemble_stream_window(g, s_list, r0, I, J, O, cap)
        tot = [a + b for a, b in zip(tot, pairs)]
    e1.record(stream)
    e1.synchronize()
    all_ms = e0.elapsed_time(e1)
    fs = slg.slg_ensemble_fill_stats(g, reset=True)
    if made is not None:
        for t, s in enumerate(s_list):
            acc = made.setdefault(s, [0] * 6)
            for c in range(6):
                acc[c] += int(fs[t][c])
    if mode_work is not None:  # per-handler work of every list (runs their count)
        for t, s in enumerate(s_list):
            mode_work[s] = slg.slg_ensemble_mode_stats(g, s_list, t)
    filt_ms = [fs[t][4] / 1e3 for t in range(len(s_list))]
    for t, s in enumerate(s_list):
        d = per_s.setdefault(s, {"s": s, "wedges": wedges[s], "pairs": tot[t], "ms": [],
                                 "fill_ms": [], "count_ms_shared": [], "filter_ms": []})
        ms = filt_ms[t] if t else all_ms - sum(filt_ms[1:])
        d["filter_ms"].append(filt_ms[t])
        d["fill_ms"].append(ms)
        d["count_ms_shared"].append(0.0)
        d["ms"].append(ms)


def sweep_of(args):
    """(sweep, windows of every list?) for the workload: the large sweep as one-walk
    windows (its hub-pair and sparse-accumulator rows dominate and are walked
    once), the medium one as an ensemble in per-list windows; --sweep and
    --ens-windows override."""
    sweep = args.sweep or ("stream" if args.workload == "large" else "ensemble")
    ens_all = (args.ens_windows or ("all" if args.workload == "large" else "per_list")) == "all"
    return sweep, ens_all


STAGED_MODES = ("sparse", "hubpair")  # handlers whose fill kernels can stage pairs


def walk_candidates(names, mode_work, s_list, sweep, fill_made, ms_tot, ln_tot, steps):
    """Roofline candidates of a step: for each handler k and pass, (pass, k, kernel
    bytes per step, ms per step, launches per step, section 8(d) model bytes per
    step, pairs the kernel wrote per step), from the per-list handler work
    mode_work[s][k] (slg_ensemble_mode_stats columns), the walks each list took
    (fill_made[s]: windows and pairs walked, windows and pairs filtered, ...) and
    the handlers' CUDA-event totals ms_tot/ln_tot[pass][k] over `steps` steps.

    Which walks ran. Counting: an ensemble's dense handlers count every list in
    one walk, and so do its sparse-accumulator and hub-pair handlers for up to
    four lists; one-walk windows walk list 0's plan once whatever the handler;
    every other counting walk is one per list. Fill: list s is walked in the
    share of its windows that did not filter it from the list before, and its
    fill kernels write the pairs of those windows. In one-walk windows the
    sparse-accumulator and hub-pair fill kernels run as the counting pass,
    writing 5 B per pair (id and overlap byte) to the pool; their fill pass walks
    only the items the pool could not hold (not modelled).

    Returns (candidates, one_walk(k), walk_f[s])."""
    def one_walk(k):
        if sweep == "stream":
            return True
        return sweep == "ensemble" and (names[k] in ("dense", "wdense") or (
            names[k] in STAGED_MODES and len(s_list) <= 4))

    walk_f, pair_f = {}, {}
    for s in s_list:
        m = fill_made.get(s)
        wins = (m[0] + m[2]) if m else 0
        walk_f[s] = m[0] / wins if wins else 1.0
        made = (m[1] + m[3]) if m else 0
        pair_f[s] = m[1] / made if made else 1.0

    def walked(col, k, fill):
        if not fill:
            if one_walk(k):
                return mode_work[s_list[0]][k][col]
            return sum(mode_work[s][k][col] for s in s_list)
        return sum(walk_f[s] * mode_work[s][k][col] for s in s_list)

    def filled_pairs(k):
        return sum(pair_f[s] * mode_work[s][k][3] for s in s_list)

    cands = []
    for k in range(len(names)):
        for fill in (False, True):
            w, inc, nonhub = walked(1, k, fill), walked(2, k, fill), walked(4, k, fill)
            model = 4 * w + 8 * inc
            if names[k] in ("dense", "wdense"):
                # what these kernels move: adj_s entries of non-hub wedges only, one
                # 4-byte hub mask per candidate partner scanned, the row's
                # wedge-range bounds; hub wedges are popcounts and read nothing
                kern = 4 * nonhub + 4 * walked(6 if fill else 5, k, fill) + 8 * inc
            elif names[k] == "hubpair":
                # entries walked (non-hub wedges + hub-pair list hits) and their bounds
                kern = 4 * nonhub + 8 * inc
            else:
                kern = model
            pw = filled_pairs(k) if fill else 0
            if sweep == "stream" and names[k] in STAGED_MODES:
                if fill:
                    kern, model, pw = 0, 0, 0
                else:
                    kern += 5 * mode_work[s_list[0]][k][3]
                    model += 5 * mode_work[s_list[0]][k][3]
            p = 1 if fill else 0
            cands.append(("fill" if fill else "count", k, kern + 12 * pw, ms_tot[p][k] / steps,
                          ln_tot[p][k] / steps, model + 12 * pw, pw))
    return cands, one_walk, walk_f


def bench_ours(args):
    import torch
    import paper_2201_11326_gb300 as slg

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.cuda.current_device()
    h, s_list, wl_text, metric, cpu_rows = workload_spec(args)
    sweep, ens_all = sweep_of(args)
    # inputs resident in HBM before the timed region
    off_d = torch.from_numpy(h.off).to(dev)
    idx_d = torch.from_numpy(h.idx).to(dev)
    stream = torch.cuda.Stream(dev)
    wedges = {}
    if sweep in ("ensemble", "stream"):
        # W_s of every s (the metric's work), outside the timed region
        with torch.cuda.stream(stream):
            g0 = slg.slg_load(off_d, idx_d, h.m, h.n, stream=stream)
            for s in s_list:
                wedges[s] = slg.slg_count(g0, s)[1]
            g0.free()
    I = torch.empty(args.window, dtype=torch.int32, device=dev)
    J = torch.empty_like(I)
    O = torch.empty_like(I)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)

    def step(per_s, timing=False, mode_work=None):
        with torch.cuda.stream(stream):
            flush.fill_(0)  # L2 flush: a 512 MiB write
            g = slg.slg_load(off_d, idx_d, h.m, h.n, stream=stream)
            if timing:
                slg.slg_set_timing(g, True)
            if sweep == "ensemble":
                run_sweep_ensemble(slg, g, s_list, (I, J, O), stream, per_s, wedges, mode_work,
                                   all_lists=ens_all, made=fill_made if timing else None)
            elif sweep == "stream":
                run_sweep_stream(slg, g, s_list, (I, J, O), stream, per_s, wedges, mode_work,
                                 made=fill_made if timing else None)
            else:
                run_sweep(slg, g, s_list, (I, J, O), stream, per_s, mode_work)
            ks = slg.slg_kernel_stats(g) if timing else None
            g.free()
        return ks

    # per-handler work of the sweep (for the roofline's algorithmic bytes),
    # recorded during the last warm-up step (or the first timed one)
    mode_work = {}
    fill_made = {}  # per s over the timed steps: windows/pairs walked, windows/pairs filtered
    for w in range(args.warmup):
        step({}, mode_work=mode_work if w == args.warmup - 1 else None)

    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = Clocks(dev)
    launches0 = slg.slg_kernel_launches()
    per_s = {}
    kstats = []
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t_start.record(stream)
    for k in range(args.steps):
        kstats.append(step(per_s, timing=True,
                           mode_work=mode_work if (k == 0 and not mode_work) else None))
    t_end.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    launches = slg.slg_kernel_launches() - launches0
    elapsed_ms = t_start.elapsed_time(t_end)
    if dist:
        t = torch.tensor([elapsed_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms = float(t.item())

    W = sum(d["wedges"] for d in per_s.values())
    P = sum(d["pairs"] for d in per_s.values())
    sec = elapsed_ms / 1e3
    value = world * W * args.steps / sec
    edges = world * P * args.steps / sec

    # roofline of the dominant kernel (dense-tile handler, counting or fill)
    import json as _json
    peaks = {}
    try:
        peaks = _json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    NM = slg.NMODES
    ms_tot = [[0.0] * NM, [0.0] * NM]
    ln_tot = [[0] * NM, [0] * NM]
    for ms, ln in kstats:
        for p in range(2):
            for k in range(NM):
                ms_tot[p][k] += ms[p][k]
                ln_tot[p][k] += ln[p][k]

    names = list(slg.MODE_NAMES)
    cands, one_walk, walk_f = walk_candidates(names, mode_work, s_list, sweep, fill_made,
                                              ms_tot, ln_tot, args.steps)
    staged = STAGED_MODES
    dom = max(cands, key=lambda c: c[3])
    # the kernel as ncu names it
    fill_flag = "1" if dom[0] == "fill" or (sweep == "stream" and names[dom[1]] in staged) else "0"
    # (the dense, sparse-accumulator and hub-pair kernels carry a second, ensemble flag)
    kname = (f"k_{names[dom[1]]}_items<{fill_flag}, 0>"
             if names[dom[1]] in ("dense", "wdense", "sparse", "hubpair")
             else f"k_{names[dom[1]]}_items<{fill_flag}>")
    dsec = dom[3] / 1e3
    achieved = dom[2] / dsec / 1e9 if dom[3] > 0 else 0.0
    model_gbs = dom[5] / dsec / 1e9 if dom[3] > 0 else 0.0
    nl = max(dom[4], 1)
    pairs_per_launch = dom[6] / nl
    traffic = profiled_traffic(kname, dom[2] / nl, pairs_per_launch)
    ms_launch = dom[3] / nl
    dram_gbs = traffic / (ms_launch / 1e3) / 1e9 if traffic and ms_launch > 0 else None
    # the output writes alone: 12 B per pair of the dominant kernel's handler
    write_gbs = (12 * dom[6] / dsec / 1e9 if dom[0] == "fill" and dom[3] > 0 else None)
    frac = achieved / hbm_peak
    roofline = {"bound": "hbm", "kernel": kname, "achieved": round(achieved, 1),
                "peak": hbm_peak, "peak_source": peak_src, "unit": "GB/s",
                "frac": round(frac, 4), "traffic": traffic,
                "bytes_per_launch": int(dom[2] / nl),
                "launches_per_step": dom[4],
                "ms_per_launch": round(ms_launch, 3),
                "kernel_share_of_step": round(dom[3] / (elapsed_ms / args.steps), 4),
                "model": ("kernel bytes (its fill kernel run as the counting pass of one-walk "
                          "windows): 4 B per entry walked (non-hub wedges and hub-pair list hits, "
                          "or wedges for the sparse accumulator) + 8 B/incidence + 5 B per pair "
                          "staged (id and overlap byte)"
                          if sweep == "stream" and names[dom[1]] in staged else
                          "kernel bytes: 12 B/pair written + 4 B per non-hub wedge (adj_s entry) "
                          "+ 4 B per candidate partner scanned (hub mask) + 8 B per incidence "
                          "(wedge-range bounds)" if names[dom[1]] in ("dense", "wdense") else
                          "kernel bytes: 4 B per entry walked (non-hub wedges and hub-pair list "
                          "hits) + 8 B/incidence + 12 B/pair written" if names[dom[1]] == "hubpair"
                          else "kernel bytes: 4 B/wedge + 8 B/incidence + 12 B/pair written"),
                "walks": ("one-walk windows: sparse-accumulator and hub-pair rows walked once "
                          "(counting and staging list 0); table and dense rows counted once before "
                          "the windows and filled in them; later lists filtered"
                          if sweep == "stream" else
                          "one counting walk for every list where the ensemble counts them "
                          "together; fill walks only of the windows that walked the list (the "
                          "others filter it from the list before)"),
                "frac_above_1": frac > 1.0,
                "alg_model_GBps": round(model_gbs, 1),
                "alg_model_frac": round(model_gbs / hbm_peak, 4),
                "alg_model": "section 8(d) model: 4 B/wedge + 8 B/incidence + 12 B/pair written "
                             "(charges hub wedges that the dense handlers never read)",
                "output_write_GBps": round(write_gbs, 1) if write_gbs else None,
                "output_write_frac": round(write_gbs / hbm_peak, 4) if write_gbs else None,
                "pairs_per_launch": int(pairs_per_launch),
                "dram_GBps": round(dram_gbs, 1) if dram_gbs else None,
                "dram_frac": round(dram_gbs / hbm_peak, 4) if dram_gbs else None}
    kernels_ms = {f"{ps}_{names[k]}": round(ms_tot[pi][k] / args.steps, 1)
                  for pi, ps in enumerate(("count", "fill")) for k in range(NM)}

    per_s_out = []
    for s in s_list:
        d = per_s[s]
        ms = statistics.mean(d["ms"])
        pw = mode_work[s]
        # walks charged to s: its share of the counting walks, its fill walks,
        # and, where it was filtered, the 12 B/pair read of the list before
        walk = [4 * pw[k][1] + 8 * pw[k][2] for k in range(NM)]
        cnt = sum(walk[k] / len(s_list) if one_walk(k) else walk[k] for k in range(NM))
        filt_read = 12 * fill_made[s][5] / args.steps if s in fill_made else 0
        alg = cnt + walk_f[s] * sum(walk) + 12 * d["pairs"] + filt_read
        rec = {"s": s, "wedges": d["wedges"], "pairs": d["pairs"],
               "ms": round(ms, 2), "wedges_per_s": d["wedges"] / (ms / 1e3),
               "s_edges_per_s": d["pairs"] / (ms / 1e3),
               "output_write_GBps": round(12 * d["pairs"] / (ms / 1e3) / 1e9, 1),
               "alg_model_GBps": round(alg / (ms / 1e3) / 1e9, 1)}
        if "fill_ms" in d:
            rec["fill_ms"] = round(statistics.mean(d["fill_ms"]), 2)
            rec["count_ms_shared"] = round(statistics.mean(d["count_ms_shared"]), 2)
        m = fill_made.get(s)
        if m and m[2]:
            # the list filter that made s from the list before: 12 B read per pair
            # of that list in the filtered windows, 12 B written per pair kept
            fbytes = 12 * m[5] + 12 * m[3]
            fsec = m[4] / 1e6
            rec["filter"] = {"windows": m[2] // args.steps, "pairs": m[3] // args.steps,
                             "ms": round(m[4] / 1e3 / args.steps, 2),
                             "GBps": round(fbytes / fsec / 1e9, 1) if fsec > 0 else None,
                             "frac": round(fbytes / fsec / 1e9 / hbm_peak, 4) if fsec > 0 else None}
        per_s_out.append(rec)

    out = {
        "metric": metric, "value": value, "unit": "wedges/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": wl_text, "sweep": sweep,
                   "ensemble_windows": (("all lists per window, later lists filtered from the "
                                         "one before where that reads less") if ens_all else
                                        "each list in its own windows") if sweep == "ensemble"
                   else ("one-walk windows of every list (rows chosen from a bound on their "
                         "pairs), later lists filtered from the one before") if sweep == "stream"
                   else None,
                   "m": h.m, "n": h.n, "nnz": h.nnz, "s": s_list, "window_pairs": args.window,
                   "l2": "flushed before each step (512 MiB device write); inputs resident",
                   "parallelism": f"replicas x{world}"},
        "s_edges_per_s": edges,
        "per_s": per_s_out,
        "kernel_ms_per_step": kernels_ms,
        "roofline": roofline,
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    if rank == 0 and not args.no_e2e:
        out["e2e"] = e2e(args, slg, h, s_list, stream, (I, J, O), sweep, all_lists=ens_all)
    if rank == 0 and world == 1 and not args.no_cpu:
        wedges, dt, cores, sample = oracle_sample(h, s_list, cpu_rows, seed=1)
        out["cpu_baseline"] = {"value": wedges / dt, "unit": "wedges/s", "cores": cores,
                               "kind": "oracle", "sample": sample, "seconds": round(dt, 2)}
    if dist:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


def e2e(args, slg, h, s_list, stream, bufs, sweep="per_s", all_lists=False):
    """Same sweep through the public API from pinned host memory (an ensemble in
    the same windows as the device-timed step: each list's own, or windows of
    every list).

    Timed (wall clock): host->device copy of the CSR (inside slg_load), the
    transpose, every counting pass and window fill, and the device->host read
    of each s-line graph's row offsets (rowoff[m+1], int64) -- the lists stay in
    the device window.
    """
    import torch
    off_h = torch.from_numpy(h.off).pin_memory()
    idx_h = torch.from_numpy(h.idx).pin_memory()
    rowoff = torch.empty(h.m + 1, dtype=torch.int64).pin_memory()
    I, J, O = bufs
    WINDOW = I.numel()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    W = 0
    with torch.cuda.stream(stream):
        g = slg.slg_load(off_h, idx_h, h.m, h.n, stream=stream)
        if sweep == "stream":
            nwin, r0 = 0, 0
            tot = [0] * len(s_list)
            while r0 < h.m:  # |L_s| of every list comes back with each window
                r0, pairs = slg.slg_ensemble_stream_window(g, s_list, r0, I, J, O, WINDOW)
                tot = [a + b for a, b in zip(tot, pairs)]
                nwin += 1
        elif sweep == "ensemble":
            slg.slg_ensemble_count(g, s_list)
            rows = torch.empty((len(s_list), h.m + 1), dtype=torch.int64).pin_memory()
            for t in ([slg.ENSEMBLE_ALL] if all_lists else range(len(s_list))):
                splits = slg.slg_ensemble_plan_windows(g, s_list, WINDOW, which=t)
                for r0, r1 in zip(splits[:-1], splits[1:]):
                    slg.slg_ensemble_build_window(g, s_list, int(r0), int(r1), I, J, O, WINDOW,
                                                  which=t)
            slg.slg_ensemble_row_offsets(g, s_list, rows)
        else:
            for s in s_list:
                splits = slg.slg_plan_windows(g, s, WINDOW)
                for r0, r1 in zip(splits[:-1], splits[1:]):
                    slg.slg_build_window(g, s, int(r0), int(r1), I, J, O, WINDOW)
                slg.slg_row_offsets(g, s, rowoff)
        g.free()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    # the metric's work, W = sum over s of W_s (counted outside the timed region)
    with torch.cuda.stream(stream):
        g = slg.slg_load(h.off, h.idx, h.m, h.n, stream=stream)
        W = sum(slg.slg_count(g, s)[1] for s in s_list)
        g.free()
    if sweep == "stream":
        return {"value": W / dt, "unit": "wedges/s",
                "h2d_bytes_per_step": int(h.off.nbytes + h.idx.nbytes),
                "d2h_bytes_per_step": int(nwin * (4 + 8 * len(s_list))), "seconds": round(dt, 3),
                "note": "lists stay in the device window; host reads each window's end and "
                        "pairs per list (|L_s| summed)"}
    return {"value": W / dt, "unit": "wedges/s", "h2d_bytes_per_step": int(h.off.nbytes + h.idx.nbytes),
            "d2h_bytes_per_step": int(8 * (h.m + 1) * len(s_list)), "seconds": round(dt, 3),
            "note": "lists stay in the device window; host reads |L_s| and row offsets"}


def kernel_source_sha(kname: str) -> str:
    """Hash of the code a kernel is built from, comments and blank lines left out:
    for the warp dense handler, its section of count_fill.cu (from its section
    banner to the next one) and the shared device helpers; for any other kernel,
    all of count_fill.cu."""
    csrc = os.path.join(ROOT, "paper_2201_11326_gb300", "csrc")
    text = open(os.path.join(csrc, "count_fill.cu"), "rb").read()
    if kname.startswith("k_wdense_items"):
        a = text.index(b"// " + b"=" * 58 + b" MODE_WDENSE")
        b = text.index(b"\n// =", a + 1)
        text = text[a:b] + open(os.path.join(csrc, "kernel_util.cuh"), "rb").read()
    code = []
    for line in text.decode().splitlines():
        line = line.split("//", 1)[0].rstrip()
        if line:
            code.append(line)
    return hashlib.sha256("\n".join(code).encode()).hexdigest()[:16]


def profiled_traffic(kname: str, alg_bytes_per_launch: float, pairs_per_launch: float):
    """DRAM bytes per launch from the committed ncu summary, if it matches.

    profiles/traffic.json maps kernel name -> the DRAM bytes the kernel moved
    per output pair on the captured case ("dram_per_pair"; its DRAM bytes are
    the output writes, so they grow with the pairs written) or, for older
    records, per algorithmic byte ("dram_over_alg"), and "source_sha", the
    hash of the kernel source when captured. Scaled to this launch; null when
    no capture exists or the kernel's source (kernel_source_sha) has changed.
    """
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path)).get(kname)
    except (OSError, ValueError):
        return None
    if not rec:
        return None
    if rec.get("source_sha") != kernel_source_sha(kname):
        return None
    if "dram_per_pair" in rec:
        return int(rec["dram_per_pair"] * pairs_per_launch)
    return int(rec["dram_over_alg"] * alg_bytes_per_launch)


# ----------------------------------------------------------- reference arm

def bench_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    h, s_list, wl_text, metric, cpu_rows = workload_spec(args)
    rows = max(8, cpu_rows // 4)
    for k in range(args.warmup):
        oracle_sample(h, s_list, rows, seed=100 + k)
    W = 0
    T = 0.0
    for k in range(args.steps):
        w, dt, cores, sample = oracle_sample(h, s_list, rows, seed=200 + k)
        W += w
        T += dt
    value = W / T
    out = {
        "impl": "reference", "metric": metric, "value": value, "unit": "wedges/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": T / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": wl_text, "m": h.m, "n": h.n, "nnz": h.nnz, "s": s_list,
                   "parallelism": "cpu oracle, host threads"},
        "cpu_baseline": {"value": value, "unit": "wedges/s", "cores": cores, "kind": "oracle",
                         "sample": f"{rows} random rows per step x s={s_list[0]}..{s_list[-1]}"},
        "e2e": {"value": value, "unit": "wedges/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------ batched form

BATCH_WORKLOAD = ("batched: {k} hypergraphs, m log-uniform in [100, 100000], n = m/2, sizes "
                  "log-normal(1.8,1.0) clipped [2,5000], Zipf(1.7) popularity, each with s "
                  "uniform in {{1,2,3,4}}")


def bench_batch(args):
    """One batch handle (disjoint union, per-graph s) against sequential calls.

    Both arms start from the same graphs already loaded on the device (inputs
    resident). Batched step: slg_batch_load + one counting pass + the fill of
    every window of the concatenated list. Sequential step: for each graph its
    own counting pass and window fills.
    """
    import torch
    import paper_2201_11326_gb300 as slg
    dev = torch.cuda.current_device()
    k = args.graphs
    t0 = time.perf_counter()
    members = [synth.batch_member(b) for b in range(k)]
    gen_s = time.perf_counter() - t0
    stream = torch.cuda.Stream(dev)
    graphs = [slg.slg_load(h.off, h.idx, h.m, h.n, stream=stream) for h, _ in members]
    s_list = [s for _, s in members]
    I = torch.empty(args.window, dtype=torch.int32, device=dev)
    J = torch.empty_like(I)
    O = torch.empty_like(I)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)

    tuned_bins = None

    def batched():
        b = slg.slg_batch_load(graphs, s_list, stream=stream)
        if tuned_bins is not None:
            slg.slg_set_bins(b, *tuned_bins)
        pairs, wedges = slg.slg_count(b, 0)
        for r0, r1 in zip(*(lambda sp: (sp[:-1], sp[1:]))(slg.slg_plan_windows(b, 0, args.window))):
            slg.slg_build_window(b, 0, int(r0), int(r1), I, J, O, args.window)
        b.free()
        return pairs, wedges

    def sequential():
        P = W = 0
        for g, s in zip(graphs, s_list):
            pairs, wedges = slg.slg_count(g, s)
            P += pairs
            W += wedges
            sp = slg.slg_plan_windows(g, s, args.window)
            for r0, r1 in zip(sp[:-1], sp[1:]):
                slg.slg_build_window(g, s, int(r0), int(r1), I, J, O, args.window)
        return P, W

    def timed(fn):
        with torch.cuda.stream(stream):
            flush.fill_(0)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            l0 = slg.slg_kernel_launches()
            e0.record(stream)
            out = fn()
            e1.record(stream)
            e1.synchronize()
        return out, e0.elapsed_time(e1), slg.slg_kernel_launches() - l0

    # the autotuner picks the batch's binning once (outside the timed steps)
    with torch.cuda.stream(stream):
        b = slg.slg_batch_load(graphs, s_list, stream=stream)
        t0 = time.perf_counter()
        tuned, tuned_ms = slg.slg_autotune(b, 0, max_trials=24)
        tune_s = time.perf_counter() - t0
        b.free()
    res = {}
    clocks = Clocks(dev)
    for name, fn in (("batched", batched), ("sequential", sequential), ("batched_autotuned", batched)):
        if name == "batched_autotuned":
            tuned_bins = tuned
        for _ in range(args.warmup):
            timed(fn)
        times, launches = [], 0
        for _ in range(args.steps):
            (P, W), ms, nl = timed(fn)
            times.append(ms)
            launches = nl
        ms = statistics.mean(times)
        res[name] = {"wedges_per_s": W / (ms / 1e3), "s_edges_per_s": P / (ms / 1e3),
                     "ms_per_step": round(ms, 1), "gpu_launches": int(launches),
                     "pairs": P, "wedges": W}
    clk = clocks.stop()
    for g in graphs:
        g.free()
    out = {
        "metric": "batched s-line wedges/s (per-graph s, one batch handle, autotuned bins)",
        "value": res["batched_autotuned"]["wedges_per_s"], "unit": "wedges/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": res["batched_autotuned"]["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": BATCH_WORKLOAD.format(k=k), "graphs": k,
                   "rows": int(sum(h.m for h, _ in members)),
                   "nnz": int(sum(h.nnz for h, _ in members)), "window_pairs": args.window,
                   "generation_s": round(gen_s, 1)},
        "batched": res["batched"], "sequential": res["sequential"],
        "batched_autotuned": dict(res["batched_autotuned"], bins=tuned, tuning_s=round(tune_s, 1)),
        "speedup_vs_sequential": (res["batched_autotuned"]["wedges_per_s"]
                                  / res["sequential"]["wedges_per_s"]),
        "clocks": clk,
    }
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------- ensemble

def run_ensemble(slg, g, s_list, bufs, strategy="all_lists"):
    """Algorithm 3 on a loaded graph: one plan for min(s_list) and one counting
    pass for every list, then the fills. "all_lists": windows hold every list of
    their rows (filled one list after another); "per_list": each list's own
    windows, filled from the shared plan one list at a time."""
    I, J, O = bufs
    cap = I.numel()
    pairs, _ = slg.slg_ensemble_count(g, s_list)
    if strategy == "all_lists":
        splits = slg.slg_ensemble_plan_windows(g, s_list, cap)
        for r0, r1 in zip(splits[:-1], splits[1:]):
            slg.slg_ensemble_build_window(g, s_list, int(r0), int(r1), I, J, O, cap)
    else:
        for t in range(len(s_list)):
            splits = slg.slg_ensemble_plan_windows(g, s_list, cap, which=t)
            for r0, r1 in zip(splits[:-1], splits[1:]):
                slg.slg_ensemble_build_window(g, s_list, int(r0), int(r1), I, J, O, cap, which=t)
    return pairs


ENSEMBLE_STRATEGY = "per_list"   # the faster fill strategy on the medium workload
OTHER_STRATEGY = "all_lists"


def bench_ensemble(args):
    """The s sweep of the medium workload as one ensemble against one s at a time.

    Both arms start from the CSR resident in HBM and run slg_load inside the
    step. Ensemble step: one plan for the smallest s, the counting pass for
    every s, then the fill of every window of all lists. Per-s step: the
    default benchmark's step. Same metric (sum over s of W_s per second).
    """
    import torch
    import paper_2201_11326_gb300 as slg
    dev = torch.cuda.current_device()
    s_list = s_values(args.s)
    h = workload(args.m)
    off_d = torch.from_numpy(h.off).to(dev)
    idx_d = torch.from_numpy(h.idx).to(dev)
    stream = torch.cuda.Stream(dev)
    I = torch.empty(args.window, dtype=torch.int32, device=dev)
    J = torch.empty_like(I)
    O = torch.empty_like(I)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    g = slg.slg_load(off_d, idx_d, h.m, h.n, stream=stream)
    counts = {s: slg.slg_count(g, s) for s in s_list}
    g.free()
    W = sum(w for _, w in counts.values())
    P = sum(p for p, _ in counts.values())

    def ens(strategy):
        def run():
            g = slg.slg_load(off_d, idx_d, h.m, h.n, stream=stream)
            slg.slg_set_timing(g, True)
            pairs = run_ensemble(slg, g, s_list, (I, J, O), strategy)
            ks = slg.slg_kernel_stats(g)
            g.free()
            assert pairs == [counts[s][0] for s in s_list]
            return ks
        return run

    def sweep():
        g = slg.slg_load(off_d, idx_d, h.m, h.n, stream=stream)
        slg.slg_set_timing(g, True)
        run_sweep(slg, g, s_list, (I, J, O), stream, {})
        ks = slg.slg_kernel_stats(g)
        g.free()
        return ks

    def timed(fn):
        with torch.cuda.stream(stream):
            flush.fill_(0)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            l0 = slg.slg_kernel_launches()
            e0.record(stream)
            ks = fn()
            e1.record(stream)
            e1.synchronize()
        return e0.elapsed_time(e1), slg.slg_kernel_launches() - l0, ks

    names = list(slg.MODE_NAMES)
    res = {}
    clocks = None
    for name, fn in (("ensemble", ens(ENSEMBLE_STRATEGY)), ("ensemble_" + OTHER_STRATEGY,
                                                           ens(OTHER_STRATEGY)),
                     ("per_s", sweep)):
        for _ in range(args.warmup):
            timed(fn)
        if name == "ensemble":
            clocks = Clocks(dev)
        times, launches, kms = [], 0, {}
        for _ in range(args.steps):
            ms, nl, (kt, _) = timed(fn)
            times.append(ms)
            launches = nl
            for pi, ps in enumerate(("count", "fill")):
                for k in range(slg.NMODES):
                    key = f"{ps}_{names[k]}"
                    kms[key] = kms.get(key, 0.0) + kt[pi][k] / args.steps
        if name == "ensemble":
            clk = clocks.stop()
        ms = statistics.mean(times)
        res[name] = {"wedges_per_s": W / (ms / 1e3), "s_edges_per_s": P / (ms / 1e3),
                     "ms_per_step": round(ms, 1), "gpu_launches": int(launches),
                     "kernel_ms_per_step": {k: round(v, 1) for k, v in kms.items()}}
    out = {
        "metric": "s-line wedges/s of an ensemble (medium hypergraph, s=1..8 as one ensemble, "
                  "bit-exact)",
        "value": res["ensemble"]["wedges_per_s"], "unit": "wedges/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": res["ensemble"]["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "m": h.m, "n": h.n, "nnz": h.nnz, "s": s_list,
                   "window_pairs": args.window, "wedges": W, "pairs": P,
                   "l2": "flushed before each step (512 MiB device write); inputs resident"},
        "strategy": ENSEMBLE_STRATEGY, "ensemble": res["ensemble"],
        "ensemble_" + OTHER_STRATEGY: res["ensemble_" + OTHER_STRATEGY], "per_s": res["per_s"],
        "speedup_vs_per_s": res["ensemble"]["wedges_per_s"] / res["per_s"]["wedges_per_s"],
        "clocks": clk,
    }
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------- served form

SERVE_WORKLOAD = ("served: 64 resident hypergraphs (8 with m=1,000,000, 56 with m log-uniform "
                  "in [1e3,1e5]; n = m/2; medium recipe), queries (uniform graph, s uniform in "
                  "1..16), Poisson arrivals")


def bench_serve(args):
    """Latency and throughput of the query server against one query at a time.

    For each arrival rate the same seeded query stream (args.queries queries) is
    played against the server with continuous batching, the same server without
    batching, and one worker (a one-query-at-a-time loop). Latency is submit ->
    result ready, reported overall and per size class (queries on the eight
    graphs with m = 1,000,000 and on the 56 small ones).
    """
    import torch
    import paper_2201_11326_gb300 as slg
    dev = torch.cuda.current_device()
    t0 = time.perf_counter()
    hs = [synth.served_member(g) for g in range(64)]
    gen_s = time.perf_counter() - t0
    gs = [slg.slg_load(h.off, h.idx, h.m, h.n) for h in hs]
    torch.cuda.synchronize()
    rates = [100, 1000, 10000]
    nq = args.queries
    rng = np.random.default_rng([1, 2])
    streams = {}
    for r in rates:
        gap = rng.exponential(1.0 / r, size=nq)
        streams[r] = (np.cumsum(gap) - gap[0], rng.integers(0, 64, size=nq),
                      rng.integers(1, 17, size=nq))

    def pct(x, q):
        return round(float(np.percentile(np.asarray(x), q)) / 1e3, 2) if len(x) else None

    def play(srv, ids, r):
        arr, gsel, ssel = streams[r]
        slg.slg_serve_stats(srv, reset=True)
        tickets = []
        start = time.perf_counter()
        for a, g, s in zip(arr, gsel, ssel):
            delay = start + a - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            tickets.append((slg.slg_serve_submit(srv, ids[int(g)], int(s)), int(g)))
        # collect in completion order, releasing each kept result at once (a
        # result held by the client counts against the server's memory budget)
        outstanding = list(tickets)
        lat = {"large": [], "small": []}
        batched = 0
        deadline = time.perf_counter() + 3600
        while outstanding and time.perf_counter() < deadline:
            still = []
            for t, g in outstanding:
                try:
                    res = slg.slg_serve_poll(srv, t, 0)
                except slg.SlgError as e:
                    if e.code != slg.SLG_ETIMEOUT:
                        raise
                    still.append((t, g))
                    continue
                lat["large" if g < 8 else "small"].append(res["latency_us"])
                batched += 1 if res["batch_size"] > 1 else 0
                slg.slg_serve_release(srv, t)
            outstanding = still
            if outstanding:
                time.sleep(0.002)
        if outstanding:
            raise RuntimeError(f"{len(outstanding)} queries did not finish")
        st = slg.slg_serve_stats(srv)
        allv = lat["large"] + lat["small"]
        return {"rate": r, "queries": nq, "p50_ms": pct(allv, 50), "p99_ms": pct(allv, 99),
                "mean_ms": round(st["mean_us"] / 1e3, 2),
                "large_m1M": {"queries": len(lat["large"]), "p50_ms": pct(lat["large"], 50),
                              "p99_ms": pct(lat["large"], 99)},
                "small": {"queries": len(lat["small"]), "p50_ms": pct(lat["small"], 50),
                          "p99_ms": pct(lat["small"], 99)},
                "queries_per_s": round(st["queries_per_s"], 2), "wedges_per_s": st["wedges_per_s"],
                "s_edges_per_s": st["pairs_per_s"], "span_s": round(st["span_s"], 2),
                "batched_queries": batched, "batches": st["batches"],
                "batch_overflows": st["batch_overflows"], "batch_failures": st["batch_failures"]}

    res = {}
    arms = (("served", dict(workers=8, policy=1, small_workers=2, small_wedges=2_000_000_000,
                            batch_max=8)),
            ("served_unbatched", dict(workers=8, policy=1, small_workers=2,
                                      small_wedges=2_000_000_000)),
            ("one_at_a_time", dict(workers=1, policy=0)))
    clk = {}
    for name, kw in arms:
        srv = slg.Server(memory_budget=64 << 30, window_pairs=1 << 28,
                         max_result_pairs=1 << 26, max_s=16, digest=False, **kw)
        ids = [slg.slg_serve_register(srv, g) for g in gs]
        # warm-up: a few queries
        for g in (0, 9, 20):
            t = slg.slg_serve_submit(srv, ids[g], 4)
            slg.slg_serve_poll(srv, t, 600000)
            slg.slg_serve_release(srv, t)
        clocks = Clocks(dev)
        res[name] = [play(srv, ids, r) for r in rates]
        clk[name] = clocks.stop()
        srv.close()
    for g in gs:
        g.free()
    served, loop = res["served"], res["one_at_a_time"]
    out = {
        "metric": "served p50/p99 query latency (s-line graphs of resident hypergraphs)",
        "value": served[0]["p99_ms"], "unit": "ms (p99 at 100 queries/s)", "n_gpus": 1,
        "higher_is_better": False, "dtype": "int32", "data": "synthetic",
        "config": {"workload": SERVE_WORKLOAD, "queries_per_rate": nq, "rates": rates,
                   "workers": 8, "policy": "least predicted W_s first, 2 of 8 workers for "
                   "queries with W_s <= 2e9, up to 8 such queries per batch",
                   "memory_budget_GiB": 64, "window_pairs": 1 << 28,
                   "max_result_pairs": 1 << 26, "generation_s": round(gen_s, 1),
                   "rows": int(sum(h.m for h in hs)), "nnz": int(sum(h.nnz for h in hs))},
        "served": served, "served_unbatched": res["served_unbatched"], "one_at_a_time": loop,
        "clocks": clk["served"], "clocks_by_arm": clk,
    }
    print(json.dumps(out), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        bench_reference(args)
    elif args.workload == "batch":
        bench_batch(args)
    elif args.workload == "serve":
        bench_serve(args)
    elif args.workload == "ensemble":
        bench_ensemble(args)
    elif args.workload == "large":
        bench_ours(args)
    else:
        bench_ours(args)


if __name__ == "__main__":
    main()
