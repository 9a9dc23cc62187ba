#!/usr/bin/env python3
"""Throughput of the multicanonical sweep on the eight-55-mer aggregation
workload (8 chains x 55 monomers, periodic L = 40, 16384 walkers, 8000 bins of
0.1 on [-400, 400), FP32 pairs with FP64 totals).

One step = one pass of the whole hot path over the batch:
  `sweeps_per_step` sweeps of every walker (batched sweep kernel; proposals,
  dE, acceptance, histogram, and the FP64 drift recompute every 100 sweeps by
  each walker's own move count) -> microcanonical analysis with jackknife
  errors over 16 walker blocks -> one Berg weight update.
Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle on
a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MUCA walker-moves/s and pair-evals/s (% FP32 peak), batched vs plain at ≤1e-4 rel ΔE"
WORKLOAD = "8x55-mer aggregation: 8 chains x 55 monomers, periodic L=40, 16384 walkers, 8000 bins of 0.1 on [-400,400)"
N_JK = 16
N_T = 64
GEOM_WALKERS = 16384
GEOM_SWEEPS = 100
FLOPS_OPEN, FLOPS_PBC = 14, 23          # algorithmic flops of one pair evaluation (open / minimum image)
LAUNCHES_PER_STEP = 5                   # sweep, 3 analysis kernels, Berg update
MOVE_NAMES = ("pivot", "translation", "rotation", "crankshaft", "bond", "cap")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--sweeps-per-step", type=int, default=10)
    ap.add_argument("--walkers", type=int, default=16384)
    ap.add_argument("--recompute-every", type=int, default=None,
                    help="sweeps between FP64 full-energy recomputes (default: the workload's)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-grad", action="store_true")
    ap.add_argument("--no-geom", action="store_true")
    ap.add_argument("--geom-only", action="store_true")
    ap.add_argument("--geom-tile", type=int, nargs=2, default=None, metavar=("TPW", "WPC"))
    ap.add_argument("--geom-walkers", type=int, default=GEOM_WALKERS)
    ap.add_argument("--eager", action="store_true",
                    help="run the headline step's sweeps and Berg update as separate calls instead of a captured "
                         "CUDA graph (always so with more than one rank: the histogram all-reduce sits between them)")
    ap.add_argument("--no-uneven", action="store_true")
    ap.add_argument("--uneven-only", action="store_true")
    ap.add_argument("--no-small", action="store_true", help="skip the 13-mer and four-9-mer workloads")
    ap.add_argument("--dry-run-cpu", action="store_true",
                    help="rank plumbing only, on CPU over gloo: walker keys, one histogram exchange per step, "
                         "max-over-ranks time (no GPU, no sweep)")
    return ap.parse_args()


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.dev), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------
# CPU oracle legs (the oracle is the reference arm and the CPU baseline)
# ----------------------------------------------------------------------------
def oracle_walker_moves_per_s(s, seconds: float, threads: int):
    """Time the FP64 oracle on a bounded sample: `threads` threads, each walker k
    sweeps (k = 1 unless one sweep is under 10 ms, so that small systems are not
    timed on the thread pool's per-task overhead).  Returns walker-moves/s,
    pair-evals/s, walkers, seconds and k."""
    from concurrent.futures import ThreadPoolExecutor

    import numpy as np

    import oracle
    m = oracle.Model(s.chain_len, s.seq, box_L=s.box_L, k_bend=s.k_bend, k_tors=s.k_tors,
                     k_lj_intra=s.k_lj_intra, k_lj_inter=s.k_lj_inter, C=s.C, sphere_R=s.sphere_R,
                     k_fene=s.k_fene, fene_r0=s.fene_r0, fene_R=s.fene_R, C_F=s.C_F)
    mu = oracle.Muca(s.e_min, s.bin_width, s.n_bins, p=s.p, amax=s.amax, recompute_every=s.recompute_every)
    lnW = np.zeros(s.n_bins)
    N = s.n_total

    def one(w, k=1):
        wk = oracle.new_walker(m, mu, s.xyz0, int(w))
        _, st, _ = oracle.sweep_walker(m, mu, lnW, wk, k * N)
        return st[oracle.ST_PAIR_EVALS]

    one(0)                                            # first call: library and model set-up
    t0 = time.perf_counter()
    one(0)
    per = time.perf_counter() - t0                    # one walker-sweep on one core
    k = max(1, int(0.01 / per))                       # sweeps per task
    if k > 1:
        t0 = time.perf_counter()
        one(0, k)
        per = (time.perf_counter() - t0) / k
    n = max(1, int(seconds / (per * k))) * threads    # about `seconds` of wall time on `threads` cores
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=threads) as ex:
        pev = sum(ex.map(lambda w: one(w, k), range(1, n + 1)))
    dt = time.perf_counter() - t0
    return n * k * N / dt, pev / dt, n, dt, k


def run_reference(args):
    rank = int(os.environ.get("RANK", 0))
    if rank != 0:
        return
    from paper_1702_01770_gb300 import inputs
    s = inputs.config4(walkers=1)
    threads = os.cpu_count() or 1
    per_step = max(1.0, args.cpu_seconds / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        oracle_walker_moves_per_s(s, per_step, threads)
    vals, pes, tot = [], [], 0.0
    for _ in range(args.steps):
        v, pe, n, dt, _ = oracle_walker_moves_per_s(s, per_step, threads)
        vals.append(v)
        pes.append(pe)
        tot += dt
    v = statistics.mean(vals)
    sample = f"{threads} threads, one sweep (440 moves) per walker, lnW = 0, {args.steps} steps of ~{per_step:.1f} s"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "walker-moves/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "walkers": "bounded sample", "impl": "FP64 CPU oracle"},
        "pair_evals_per_s": statistics.mean(pes),
        "cpu_baseline": {"value": v, "unit": "walker-moves/s", "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "walker-moves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------
SWEEP_SOURCES = ("common.cuh", "group.cuh", "lane.cuh", "sweep.cu")   # what the sweep kernels are compiled from


def csrc_digest() -> str:
    """Digest of the sweep kernel's sources: a committed traffic figure counts only while it matches."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1702_01770_gb300", "csrc")
    for fn in SWEEP_SOURCES:
        h.update(fn.encode())
        h.update(open(os.path.join(d, fn), "rb").read())
    return h.hexdigest()[:16]


def traffic_per_launch(walkers: int):
    """DRAM bytes of one sweep launch, from the committed ncu summary (null if the kernel changed since)."""
    p = os.path.join(ROOT, "profiles", "sweep_batched_8x55_traffic.json")
    try:
        j = json.load(open(p))
    except Exception:
        return None
    if j.get("csrc_sha") != csrc_digest():
        return None
    return j["dram_bytes_per_walker"] * walkers


def measure_geometry(args, dev, walkers=None):
    """The paper's own geometry: steric sphere, FENE bonds, bond-length and cap moves
    (the builds with them), two Fibonacci 13-mers, FP32 pair terms, on the tile the
    autotuner picks (one walker per thread or a group of lanes per walker)."""
    import torch

    from paper_1702_01770_gb300 import inputs, phast
    walkers = walkers or args.geom_walkers
    gsys = inputs.fene_sphere(walkers=walkers)
    gctx = phast.Context(gsys, pair_precision=32)
    glnW = torch.zeros(gsys.n_bins, dtype=torch.float64, device=dev)
    if args.geom_tile:
        gctx.set_tile(*args.geom_tile)
    else:
        gctx.autotune(glnW, sweeps=10)   # small chains: the best tile depends on the workload
    gtile = gctx.get_tile()
    gctx.sweep(20, glnW)
    torch.cuda.synchronize()
    g0 = gctx.stats()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    gctx.sweep(GEOM_SWEEPS, glnW)
    b.record()
    torch.cuda.synchronize()
    g1 = gctx.stats()
    gms = a.elapsed_time(b)
    gmoves = int(g1["attempts"].sum() - g0["attempts"].sum())
    assert gmoves == walkers * gsys.n_total * GEOM_SWEEPS
    res = {
        "workload": "2 Fibonacci 13-mers in a steric sphere R = 8, FENE bonds (k_F = -20, R_F = 0.3), "
                    f"all six move types, {walkers} walkers, flat weights, {GEOM_SWEEPS} sweeps",
        "kernel": ("sweep_lane_kernel<float,1> (one walker per thread)" if gtile[0] == 1
                   else f"sweep_batched_kernel<{gtile[0]},float,1>"), "tile": list(gtile),
        "walker_moves_per_s": gmoves / (gms / 1e3),
        "pair_evals_per_s": float((g1["pair_evals"].sum() - g0["pair_evals"].sum()) / (gms / 1e3)),
        "accept_rate": float((g1["accepts"].sum() - g0["accepts"].sum()) / gmoves), "dtype": "f32",
        "l2": "walker state %.0f MB, L2-resident" % (walkers * gsys.n_total * 24 / 1e6)}
    if not args.no_cpu_baseline and walkers == args.geom_walkers:
        v, pev, n, dt, k = oracle_walker_moves_per_s(inputs.fene_sphere(walkers=1), 4.0, os.cpu_count() or 1)
        res["cpu_baseline"] = {"value": v, "unit": "walker-moves/s", "cores": os.cpu_count() or 1,
                               "kind": "oracle", "sample": f"{n} walkers x {k} sweeps, FP64 oracle, "
                                                           f"{dt:.1f} s", "pair_evals_per_s": pev}
    gctx.close()
    return res


SMALL_SWEEPS = {"fib13": 10000, "4x9": 2000}   # sweeps timed per small workload


def measure_small(args, dev, peak_tf):
    """The two small workloads of the measurement table, each on its autotuned tile:
    the Fibonacci 13-mer (8 walkers, pivot moves, FP64 pairs, one Berg iteration's
    10^4 sweeps) and four 9-mers in L = 20 (256 walkers, FP32 pairs, FP64 recompute
    every 100 sweeps, 2000 of the workload's 10^5 sweeps), with the FP64 oracle
    beside each on a bounded sample of the same system."""
    import torch

    from paper_1702_01770_gb300 import inputs, phast
    out = {}
    for s, prec, label in ((inputs.config0(), 64, "Fibonacci 13-mer ABBABBABABBAB, 8 walkers, pivot only, "
                                                  "720 bins of 0.05, FP64 pairs"),
                           (inputs.config1(), 32, "four 9-mers (seed-1 sequences), L = 20, 256 walkers, "
                                                  "70/15/15 pivot/translation/rotation, FP32 pairs, FP64 totals")):
        n_sw = SMALL_SWEEPS[s.name]
        ctx = phast.Context(s, pair_precision=prec)
        lnW = ctx.lnW_zeros()
        tile = ctx.autotune(lnW, sweeps=10)
        ctx.sweep(20, lnW)
        torch.cuda.synchronize()
        s0 = ctx.stats()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        ctx.sweep(n_sw, lnW)
        b.record()
        torch.cuda.synchronize()
        s1 = ctx.stats()
        ms = a.elapsed_time(b)
        mv = int(s1["attempts"].sum() - s0["attempts"].sum())
        assert mv == s.walkers * s.n_total * n_sw
        pe = int(s1["pair_evals"].sum() - s0["pair_evals"].sum())
        pex = int(s1["pair_evals_inter"].sum() - s0["pair_evals_inter"].sum())
        r = {"workload": label, "sweeps": n_sw, "tile": list(tile), "ms": ms,
             "walker_moves_per_s": mv / (ms / 1e3), "pair_evals_per_s": pe / (ms / 1e3),
             "dtype": "f64" if prec == 64 else "f32"}
        if prec == 32:
            r["fp32_frac"] = _flops(pe, pex) / (ms / 1e3) / 1e12 / peak_tf
        ctx.close()
        if not args.no_cpu_baseline:
            v, pev, n, dt, k = oracle_walker_moves_per_s(s, 2.0, os.cpu_count() or 1)
            r["cpu_baseline"] = {"value": v, "unit": "walker-moves/s", "cores": os.cpu_count() or 1, "kind": "oracle",
                                 "sample": f"{n} walkers x {k} sweeps, FP64 oracle, {dt:.1f} s",
                                 "pair_evals_per_s": pev}
        out[s.name] = r
    return out


UNEVEN_CHUNK = 1000        # sweeps per captured iteration of the four-type workload


def _flops(pe, pex):
    return (pe - pex) * FLOPS_OPEN + pex * FLOPS_PBC


def measure_uneven(args, dev, peak_tf):
    """Four uneven system types in one persistent launch (1024 walkers each: a
    Fibonacci 13-mer, a Fibonacci 21-mer, two 34-mers in L = 40, eight 9-mers in
    L = 30), FP32 pairs: the autotuned tile, one multicanonical iteration of
    UNEVEN_CHUNK sweeps captured as a CUDA graph and replayed; then each type alone
    (its own autotuned tile) and the plain FP64 form on the same four types."""
    import numpy as np
    import torch

    from paper_1702_01770_gb300 import inputs, phast
    systems = inputs.config2(walkers_each=1024)
    ctx = phast.Context(systems, pair_precision=32)
    lnW = ctx.lnW_zeros()
    g = torch.zeros_like(lnW)
    n_jk = 16
    hs = ctx.hist_sum_zeros(n_jk)
    flat = torch.zeros(len(systems), 4, dtype=torch.float64, device=dev)
    default_tile = ctx.get_tile()
    tile = ctx.autotune(lnW, sweeps=10)
    graph = ctx.capture_iteration(UNEVEN_CHUNK, lnW, hs, g, n_jk=n_jk, flat_out=flat)
    graph.launch()                               # warm-up iteration
    torch.cuda.synchronize()
    st0 = ctx.stats()
    reps = 3
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        graph.launch()
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / reps
    st1 = ctx.stats()
    graph.close()
    per_type = []
    for k, x in enumerate(systems):
        sl = slice(ctx.walker_off[k], ctx.walker_off[k] + x.walkers)
        mv = int(st1["attempts"][sl].sum() - st0["attempts"][sl].sum()) // reps
        pe = int(st1["pair_evals"][sl].sum() - st0["pair_evals"][sl].sum()) // reps
        pex = int(st1["pair_evals_inter"][sl].sum() - st0["pair_evals_inter"][sl].sum()) // reps
        per_type.append({"system": x.name, "walkers": x.walkers, "moves_per_chunk": mv, "pair_evals_per_chunk": pe,
                         "pair_evals_inter_per_chunk": pex})
    moves = sum(t["moves_per_chunk"] for t in per_type)
    pe = sum(t["pair_evals_per_chunk"] for t in per_type)
    fl = sum(_flops(t["pair_evals_per_chunk"], t["pair_evals_inter_per_chunk"]) for t in per_type)
    ctx.close()
    # each type alone: the share of the chip it gets when it has the chip to itself
    for k, x in enumerate(systems):
        c1 = phast.Context(x, pair_precision=32)
        l1 = c1.lnW_zeros()
        t1 = c1.autotune(l1, sweeps=10)
        c1.sweep(20, l1)
        torch.cuda.synchronize()
        s0 = c1.stats()
        a.record()
        c1.sweep(200, l1)
        b.record()
        torch.cuda.synchronize()
        s1 = c1.stats()
        t_ms = a.elapsed_time(b)
        m1 = int(s1["attempts"].sum() - s0["attempts"].sum())
        p1 = int(s1["pair_evals"].sum() - s0["pair_evals"].sum())
        x1 = int(s1["pair_evals_inter"].sum() - s0["pair_evals_inter"].sum())
        per_type[k]["alone"] = {"tile": list(t1), "walker_moves_per_s": m1 / (t_ms / 1e3),
                                "pair_evals_per_s": p1 / (t_ms / 1e3),
                                "fp32_frac": _flops(p1, x1) / (t_ms / 1e3) / 1e12 / peak_tf}
        c1.close()
    res = {"workload": "four system types in one launch, 1024 walkers each: Fibonacci 13-mer, Fibonacci 21-mer, "
                       "2 x 34-mer (L = 40), 8 x 9-mer (L = 30); FP32 pairs, FP64 totals",
           "launch": f"captured CUDA graph per iteration of {UNEVEN_CHUNK} sweeps (clear, sweeps, Berg per type)",
           "tile_autotuned": list(tile), "tile_default": list(default_tile), "ms_per_chunk": ms,
           "walker_moves_per_s": moves / (ms / 1e3), "pair_evals_per_s": pe / (ms / 1e3),
           "fp32_frac": fl / (ms / 1e3) / 1e12 / peak_tf, "per_type": per_type, "dtype": "f32"}
    # the plain one-walker-per-CTA FP64 form on the same four types
    cp = phast.Context(systems, pair_precision=64)
    lp = cp.lnW_zeros()
    cp.sweep(1, lp, form=phast.FORM_PLAIN)
    torch.cuda.synchronize()
    p0 = cp.stats()
    a.record()
    cp.sweep(5, lp, form=phast.FORM_PLAIN)
    b.record()
    torch.cuda.synchronize()
    p1 = cp.stats()
    pms = a.elapsed_time(b)
    res["plain"] = {"walker_moves_per_s": float((p1["attempts"].sum() - p0["attempts"].sum()) / (pms / 1e3)),
                    "pair_evals_per_s": float((p1["pair_evals"].sum() - p0["pair_evals"].sum()) / (pms / 1e3)),
                    "sweeps": 5, "dtype": "f64"}
    res["batched_over_plain"] = res["walker_moves_per_s"] / res["plain"]["walker_moves_per_s"]
    cp.close()
    return res


def run_ours(args):
    import numpy as np
    import torch

    from paper_1702_01770_gb300 import inputs, parallel, phast

    rank, world, local = parallel.world()
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.geom_only:   # the geometry measurement alone (a profiling aid)
        if rank == 0:
            print(json.dumps({"geometry": measure_geometry(args, dev)}), flush=True)
        return
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    max_mhz = float(peaks.get("sm_max_mhz") or 2070.0)
    if args.uneven_only:   # the four-type workload alone (a profiling aid)
        if rank == 0:
            print(json.dumps({"uneven": measure_uneven(args, dev, n_sm * 256 * max_mhz * 1e6 / 1e12)}), flush=True)
        return

    s = inputs.config4(walkers=args.walkers)
    if args.recompute_every is not None:
        s.recompute_every = args.recompute_every
    s.seed_base = parallel.walker_seed_base(rank, args.walkers)
    K, N, S = s.n_bins, s.n_total, args.sweeps_per_step
    ctx = phast.Context(s, pair_precision=32)
    lnW = torch.zeros(K, dtype=torch.float64, device=dev)
    g = torch.zeros(K - 1, dtype=torch.float64, device=dev)
    flat = torch.zeros(4, dtype=torch.float64, device=dev)
    hs = torch.zeros(N_JK * K, dtype=torch.int64, device=dev)
    T = torch.linspace(0.3, 3.0, N_T, dtype=torch.float64, device=dev)
    ws = torch.empty(phast.lib().phast_micro_workspace_size(K, N_T, N_JK), dtype=torch.uint8, device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    use_graph = not args.eager and world == 1
    graph, lnW_used = None, torch.empty_like(lnW)
    if use_graph:   # one multicanonical iteration (clear, sweeps, Berg) as a captured CUDA graph
        graph = ctx.capture_iteration(S, lnW, hs, g, n_jk=N_JK, flat_out=flat)
        torch.cuda.synchronize()

    def step(i=None):
        if use_graph:
            lnW_used.copy_(lnW)            # the weights this iteration samples with (Berg rewrites lnW)
            if i is not None:
                ev[i][0].record()
            graph.launch()
            if i is not None:
                ev[i][1].record()
            return phast.phast_micro_analysis(lnW_used, s.e_min, s.bin_width, hist=hs.view(N_JK, K),
                                              fd_half_width=5, n_monomers=N, T=T, workspace=ws)
        hs.zero_()
        if i is not None:
            ev[i][0].record()
        ctx.sweep(S, lnW, n_jk=N_JK, hist_sum=hs)
        if i is not None:
            ev[i][1].record()
        parallel.combine_histograms(hs)
        res = phast.phast_micro_analysis(lnW, s.e_min, s.bin_width, hist=hs.view(N_JK, K), fd_half_width=5,
                                         n_monomers=N, T=T, workspace=ws)
        phast.phast_weight_update(hs.view(N_JK, K), lnW, g, s.bin_width, flat_out=flat)
        return res

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    st0 = ctx.stats()
    sampler = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    for i in range(args.steps):
        res = step(i)
    t1.record()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    ms_local = t0.elapsed_time(t1)
    ms = parallel.max_over_ranks(ms_local, dev)
    st1 = ctx.stats()
    moves = int(st1["attempts"].sum() - st0["attempts"].sum())
    pe = int(st1["pair_evals"].sum() - st0["pair_evals"].sum())
    pex = int(st1["pair_evals_inter"].sum() - st0["pair_evals_inter"].sum())
    assert moves == args.walkers * N * S * args.steps
    sweep_ms = [a.elapsed_time(b) for a, b in ev]
    flops = (pe - pex) * FLOPS_OPEN + pex * FLOPS_PBC
    total_moves = moves * world
    value = total_moves / (ms / 1e3)

    # roofline of the sweep kernel: algorithmic FP32 flops / its event-timed duration
    max_mhz = float(peaks.get("sm_max_mhz") or clocks.get("sm_max_mhz") or 2070.0)
    peak_tf = n_sm * 128 * 2 * max_mhz * 1e6 / 1e12
    achieved_tf = flops / (sum(sweep_ms) / 1e3) / 1e12
    roofline = {"bound": "alu", "achieved": achieved_tf, "peak": peak_tf, "unit": "TFLOP/s",
                "frac": achieved_tf / peak_tf, "traffic": traffic_per_launch(args.walkers),
                "peak_basis": f"derived: {n_sm} SMs x 128 FP32 lanes x 2 flop x {max_mhz:.0f} MHz (max SM clock)",
                "kernel": "sweep_batched_kernel<32,float,0,1> (no FENE, sphere, bond or cap moves)",
                "frac_at_median_clock": (achieved_tf / (n_sm * 256 * clocks["sm_mhz"] * 1e6 / 1e12))
                if clocks.get("sm_mhz") else None,
                "timed": ("CUDA events around each captured iteration (histogram clear, the sweep kernel, "
                          "the Berg kernel)" if use_graph else "CUDA events around each sweep launch")}

    out = {
        "metric": METRIC, "value": value, "unit": "walker-moves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "walkers_per_gpu": args.walkers, "sweeps_per_step": S,
                   "step": "sweeps + analysis (16 jackknife blocks, 64 T) + Berg update",
                   "precision": "FP32 pair and local terms, FP64 geometry/totals/weights/histogram sums",
                   "l2": "inputs larger than L2 (walker state %.0f MB)" % (args.walkers * N * 24 / 1e6),
                   "tile": list(ctx.get_tile()),
                   "launch": ("captured CUDA graph per iteration (clear, sweeps, Berg), analysis after it"
                              if use_graph else "separate calls")},
        "pair_evals_per_s": pe * world / (ms / 1e3),
        "sweep_kernel_ms_per_step": sum(sweep_ms) / args.steps,
        "roofline": roofline,
        "gpu_launches": LAUNCHES_PER_STEP * args.steps,
        "clocks": clocks,
        "drift_max": float(st1["drift_max"].max()),
        "drift_per_walker": {"p50": float(np.percentile(st1["drift_max"], 50)),
                             "p99": float(np.percentile(st1["drift_max"], 99))},
        "recompute_every": s.recompute_every,
        "recompute_outside": int(st1["recompute_outside"].sum()),
        "accept_rate": {name: (float(a) / float(n) if n else None) for name, a, n in
                        zip(MOVE_NAMES, st1["accepts"].sum(0) - st0["accepts"].sum(0),
                            st1["attempts"].sum(0) - st0["attempts"].sum(0))},
        "flatness_cvar": float(flat[2].item()),
    }

    # plain one-walker-per-CTA FP64 form, same GPU, a subset of the walkers
    if not args.no_plain and rank == 0:
        ps = inputs.config4(walkers=2432)
        pctx = phast.Context(ps, pair_precision=64)
        plnW = torch.zeros(K, dtype=torch.float64, device=dev)
        pctx.sweep(1, plnW, form=phast.FORM_PLAIN)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0 = pctx.stats()
        a.record()
        pctx.sweep(1, plnW, form=phast.FORM_PLAIN)
        b.record()
        torch.cuda.synchronize()
        p1 = pctx.stats()
        pms = a.elapsed_time(b)
        out["plain"] = {"walker_moves_per_s": float((p1["attempts"].sum() - p0["attempts"].sum()) / (pms / 1e3)),
                        "pair_evals_per_s": float((p1["pair_evals"].sum() - p0["pair_evals"].sum()) / (pms / 1e3)),
                        "walkers": 2432, "sweeps": 1, "dtype": "f64"}
        out["batched_over_plain"] = out["pair_evals_per_s"] / world / out["plain"]["pair_evals_per_s"]
        pctx.close()

    # differentiation: energy, dE/dx and dE/d(force-field parameters) of the batch of
    # 65536 random self-avoiding walks of the Fibonacci 55-mer, FP32 terms
    if not args.no_grad and rank == 0:
        gs, gx0 = inputs.config3()
        gxyz = torch.from_numpy(gx0).to(dev)
        for _ in range(2):
            phast.phast_energy_grad(gs, gxyz, 32)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 5
        a.record()
        for _ in range(reps):
            phast.phast_energy_grad(gs, gxyz, 32)
        b.record()
        torch.cuda.synchronize()
        gms = a.elapsed_time(b) / reps
        n = gs.n_total
        pairs = n * (n - 1) // 2 - (n - 1)
        # roofline: each of the `pairs` Lennard-Jones pairs of a conformation gives its energy term
        # (14 flops) and its gradient contribution (4 more for dphi/dr^2, 6 for the force on both
        # ends: 24 flops); the kernel evaluates each pair from both of its ends
        grad_tf = gx0.shape[0] * pairs * 24 / (gms / 1e3) / 1e12
        out["differentiation"] = {"workload": "65536 random self-avoiding walks of a Fibonacci 55-mer (d_min 0.8)",
                                  "ms_per_batch": gms, "conformations_per_s": gx0.shape[0] / (gms / 1e3),
                                  "pair_terms_per_s": gx0.shape[0] * pairs / (gms / 1e3),
                                  "outputs": "E, dE/dx, dE/d(C_AA, C_BB, C_AB, kappa, kappa_C)", "dtype": "f32",
                                  "roofline": {"bound": "alu", "achieved": grad_tf, "peak": peak_tf,
                                               "unit": "TFLOP/s", "frac": grad_tf / peak_tf,
                                               "kernel": "energy_grad32_chain_kernel",
                                               "flops_per_pair": 24}}
        del gxyz

    # free energy and Maxwell construction of the last step's S(E), with the
    # leave-one-block-out replicates of its 16 jackknife blocks
    if rank == 0:
        for _ in range(2):
            phast.phast_maxwell(lnW, hs.view(N_JK, K), s.e_min, s.bin_width, N, fd_half_width=5)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 10
        a.record()
        for _ in range(reps):
            phast.phast_maxwell(lnW, hs.view(N_JK, K), s.e_min, s.bin_width, N, fd_half_width=5)
        b.record()
        torch.cuda.synchronize()
        out["maxwell"] = {"ms_per_call": a.elapsed_time(b) / reps, "bins": K, "replicates": 1 + N_JK,
                          "outputs": "f(E) per monomer; beta_c, eps_1, eps_2, latent heat, barrier, with errors"}

    if not args.no_geom and rank == 0:
        out["geometry"] = measure_geometry(args, dev)
        # one walker per thread fills the chip only with tens of thousands of walkers
        out["geometry_65536"] = measure_geometry(args, dev, walkers=65536)

    if not args.no_uneven and rank == 0:
        out["uneven"] = measure_uneven(args, dev, peak_tf)

    if not args.no_small and rank == 0:
        out["small"] = measure_small(args, dev, peak_tf)

    # end to end through the C ABI with host buffers: state in from pinned host memory, results out
    if not args.no_e2e:
        st = ctx.get_state("cpu")
        torch.cuda.synchronize()
        host = {k: v.pin_memory() for k, v in st.items() if k in ("xyz", "E", "bin", "t")}
        out_host = {k: torch.empty_like(v).pin_memory() for k, v in host.items()}
        S_host = torch.empty(K, dtype=torch.float64).pin_memory()
        lnW_host = torch.empty(K, dtype=torch.float64).pin_memory()
        h2d = sum(v.numel() * v.element_size() for v in host.values())
        d2h = h2d + 2 * K * 8
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        e0 = time.perf_counter()
        for i in range(args.steps):
            ctx.set_state(xyz=host["xyz"], E=host["E"], bin=host["bin"], t=host["t"])
            res = step()
            phast._check(phast.lib().phast_ctx_get_state(ctx.h, out_host["xyz"].data_ptr(), out_host["E"].data_ptr(),
                                                         out_host["bin"].data_ptr(), out_host["t"].data_ptr(), None,
                                                         phast._stream(None)))
            S_host.copy_(res.S, non_blocking=True)
            lnW_host.copy_(lnW, non_blocking=True)
            torch.cuda.current_stream().synchronize()
            host, out_host = out_host, host
        e_ms = (time.perf_counter() - e0) * 1e3
        e_ms = parallel.max_over_ranks(e_ms, dev)
        out["e2e"] = {"value": total_moves / (e_ms / 1e3), "unit": "walker-moves/s", "h2d_bytes_per_step": h2d,
                      "d2h_bytes_per_step": d2h}

    if rank == 0 and not args.no_cpu_baseline:
        v, pev, n, dt, _ = oracle_walker_moves_per_s(inputs.config4(walkers=1), args.cpu_seconds,
                                                     os.cpu_count() or 1)
        out["cpu_baseline"] = {"value": v, "unit": "walker-moves/s", "cores": os.cpu_count() or 1, "kind": "oracle",
                               "sample": f"{n} walkers x 1 sweep (440 moves) of the 8x55-mer workload, lnW = 0, "
                                         f"FP64 oracle, {dt:.1f} s", "pair_evals_per_s": pev}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if graph is not None:
        graph.close()
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def relaunch(args) -> int:
    """`--gpus N` (N > 1) outside torchrun: start N ranks on this node, one per GPU."""
    import socket
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        port = so.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={args.gpus}",
           "--master-addr", "127.0.0.1", f"--master-port={port}", os.path.abspath(__file__), *sys.argv[1:]]
    return subprocess.call(cmd)


def run_dry(args):
    """The multi-rank plumbing of the GPU arm on CPU (gloo): each rank's walker keys,
    one histogram all-reduce per step, the max-over-ranks time; rank 0 prints one line."""
    import torch

    from paper_1702_01770_gb300 import inputs, parallel
    rank, world, _ = parallel.world()
    if world > 1:
        torch.distributed.init_process_group("gloo")
    s = inputs.config4(walkers=args.walkers)
    s.seed_base = parallel.walker_seed_base(rank, args.walkers)
    keys = s.seeds()
    K = s.n_bins
    hs = torch.zeros(N_JK * K, dtype=torch.int64)
    exchanges = 0
    t0 = time.perf_counter()
    for i in range(args.warmup + args.steps):
        hs.zero_()
        hs[(rank * 7 + i) % K] = rank + 1          # a rank-specific count, summed by the exchange
        parallel.combine_histograms(hs)
        exchanges += 1
        assert int(hs.sum()) == world * (world + 1) // 2
    local_ms = (time.perf_counter() - t0) * 1e3
    ms = parallel.max_over_ranks(local_ms, torch.device("cpu"))
    mine = torch.tensor([float(keys[0]), float(keys[-1]), local_ms], dtype=torch.float64)
    rows = [torch.zeros_like(mine) for _ in range(world)]
    if world > 1:
        torch.distributed.all_gather(rows, mine)
    else:
        rows = [mine]
    if rank == 0:
        print(json.dumps({"dry_run": True, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                          "exchanges_per_step": exchanges / (args.warmup + args.steps), "max_ms": ms,
                          "rank_ms": [float(r[2]) for r in rows],
                          "key_ranges": [[int(r[0]), int(r[1])] for r in rows], "scaling": "weak"}), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        sys.exit(relaunch(args))
    if args.impl == "reference":
        run_reference(args)
    elif args.dry_run_cpu:
        run_dry(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
